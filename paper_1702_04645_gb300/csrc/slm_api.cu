// slm_api.cu -- host driver of the Synchronised Louvain Method (Algorithm 1)
// and the C ABI declared in slm.h and slm_steps.h.
//
// Per level t (Algorithm 1):
//   ASSIGN -> COMPONENTS -> POSITIVE, then while a node has a positive move:
//   MAXIMAL (scan, branch gains, draw, target, one synchronous write) ->
//   COMPONENTS -> POSITIVE; then compaction, and AGGREGATE when the level
//   found structure (K < n).  Every step runs in the kernels of k_*.cu; the
//   host only reads the few counters that decide the control flow.
#include <algorithm>
#include <array>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "driver.cuh"
#include "slm_internal.cuh"
#include "slm_steps.h"

using slm::DevBuf;
using slm::Work;

struct slm_graph {
    int32_t n0 = 0;
    int32_t nnz0 = 0;
    long long m = 0;
    DevBuf rp, col, w, s;  // the input graph (device copies)
    // a directed graph: rp/col/w hold U = W + W^T and s2 the packed (out, in)
    // strengths (Section 2.4); s is unused
    bool directed = false;
    DevBuf s2;
    bool has_run = false;
    struct Level {
        int32_t n = 0, K = 0;
        DevBuf labels;  // ids on this level's nodes
        DevBuf comp;    // partition composed onto the input nodes
        slm_level_stats st{};
    };
    std::vector<Level> levels;
    slm_level_stats top{};
    DevBuf final_comp;
    std::vector<std::array<long long, 6>> trace;
    std::string err;
    // per-phase device time of the last run (SLM_FLAG_TIMING)
    double phase_ms[8] = {0};
    long long phase_cnt[8] = {0};
    long long pos_ns[slm::kPosPhases] = {0};  // POSITIVE round phases (SLM_FLAG_TIMING)
    // scan time and scan count per level (SLM_FLAG_TIMING); the last entry is the top level
    std::vector<std::pair<double, long long>> scan_by_level;
    double bucket_ms[slm::kNumBuckets] = {0};  // level-0 scan time per degree bucket
};

namespace {

thread_local std::string g_create_error;

// Phases timed with CUDA events on the run's stream when SLM_FLAG_TIMING is set.
enum Phase { kPhAssign = 0, kPhComponents, kPhPositive, kPhScan, kPhMove, kPhLevel, kPhSigma,
             kPhPosRounds, kNumPhases };

struct PhaseTimer {
    bool on = false;
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    double *ms = nullptr;
    long long *cnt = nullptr;
    PhaseTimer(bool enable, cudaStream_t s, double *ms_, long long *cnt_) : on(enable), st(s), ms(ms_), cnt(cnt_) {
        if (!on) return;
        SLM_CUDA(cudaEventCreate(&a));
        SLM_CUDA(cudaEventCreate(&b));
    }
    ~PhaseTimer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
    void start() {
        if (on) SLM_CUDA(cudaEventRecord(a, st));
    }
    void stop(int phase) {
        if (!on) return;
        SLM_CUDA(cudaEventRecord(b, st));
        SLM_CUDA(cudaEventSynchronize(b));
        float t = 0;
        SLM_CUDA(cudaEventElapsedTime(&t, a, b));
        ms[phase] += t;
        cnt[phase] += 1;
    }
};

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

namespace slm {
void set_global_error(const std::string &msg) { g_create_error = msg; }
}  // namespace slm

namespace {

template <class F> slm_status guarded(slm_graph *g, F &&f) {
    try {
        f();
        return SLM_OK;
    } catch (const slm::Error &e) {
        if (g) g->err = e.msg;
        else g_create_error = e.msg;
        return e.status;
    } catch (const std::exception &e) {
        if (g) g->err = e.what();
        else g_create_error = e.what();
        return SLM_ERR_CUDA;
    }
}

__global__ void k_iota(int32_t n, int32_t *p) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = (int32_t)i;
}
__global__ void k_fill_ones(long long n, int32_t *p) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = 1;
}

// POSITIVE until no community holds a node with a negative local gain.
template <class NM>
long long positive_all(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                       const typename NM::ST *s, long long m, Work &W, cudaStream_t st,
                       PhaseTimer *tm = nullptr, bool since_last = false) {
    if (tm) tm->start();
    long long rounds = 0, visits = 0;
    long long splits = slm::positive_correct<NM>(n, rp, col, w, s, m, W.a.as<int32_t>(), W.f,
                                             W.sigma.as<typename NM::ST>(), W.bk, W.ps, st, &rounds,
                                             &visits, nullptr,
                                             since_last ? W.prev_root.as<int32_t>() : nullptr);
    if (tm) {
        tm->stop(kPhPositive);
        tm->ms[kPhPosRounds] += (double)visits;
        tm->cnt[kPhPosRounds] += rounds;
    }
    return splits;
}

struct SweepCounts {
    long long cand = 0, pos = 0, acc = 0;
};

// One MAXIMAL correction: scan, branch gains, draw, target, write.
template <class NM>
SweepCounts maximal_once(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                         const typename NM::ST *s, long long m, Work &W, unsigned long long seed,
                         unsigned long long P, int level, int sweep,
                         cudaStream_t st, slm::HostCounters &hc, PhaseTimer *tm = nullptr) {
    SweepCounts c;
    unsigned long long *ctr = W.ctr();
    if (tm) tm->start();
    SLM_CUDA(cudaMemsetAsync(ctr, 0, 64, st));
    using ST = typename NM::ST;
    slm::community_sigma(n, W.f.root, s, W.sigma.as<ST>(), st);
    if (tm) tm->stop(kPhSigma);
    if (tm) tm->start();
    slm::scan_nodes<NM>(n, rp, col, w, s, m, W.f.root, W.sigma.as<ST>(), W.bk,
                    W.best.as<int32_t>(), W.gain.as<long long>(), W.kown.as<int32_t>(), ctr, st);
    if (tm) tm->stop(kPhScan);
    if (tm) tm->start();
    // branch gains and the draw are queued before the candidate count is
    // read: with no candidate they find nothing to accept, and the host waits
    // once per sweep instead of twice
    slm::branch_gains<NM>(n, rp, col, w, s, m, W.a.as<int32_t>(), W.f, W.sigma.as<ST>(),
                      W.best.as<int32_t>(), W.gain.as<long long>(), W.kown.as<int32_t>(), W.bs,
                      W.bg.as<long long>(), st);
    int32_t *acc_cnt = reinterpret_cast<int32_t *>(ctr + 2);
    slm::accept_moves(n, W.bg.as<long long>(), seed, P, level, sweep, W.acclist.as<int32_t>(),
                      acc_cnt, ctr + 1, st);
    SLM_CUDA(cudaMemcpyAsync(hc.h, ctr, 24, cudaMemcpyDeviceToHost, st));
    slm::stream_sync(st);
    c.cand = (long long)hc.h[0];
    c.pos = (long long)hc.h[1];
    c.acc = (long long)(int32_t)(hc.h[2] & 0xffffffff);
    if (c.cand == 0 || c.pos == 0 || c.acc == 0) {
        if (tm) tm->stop(kPhMove);
        return c;
    }
    slm::target_nodes<NM>(W.acclist.as<int32_t>(), acc_cnt, (int32_t)c.acc, rp, col, w, s, m,
                      W.f.root, W.best.as<int32_t>(), W.tgt.as<int32_t>(), st);
    slm::apply_moves(W.acclist.as<int32_t>(), acc_cnt, (int32_t)c.acc, W.tgt.as<int32_t>(),
                     W.a.as<int32_t>(), st);
    if (tm) tm->stop(kPhMove);
    return c;
}

template <class NM>
void run_impl(slm_graph *g, const slm_options &opt, cudaStream_t st) {
    using ST = typename NM::ST;
    if (opt.max_sweeps < 0 || opt.max_sweeps > 65535 || opt.max_levels < 0 ||
        opt.max_levels > 65535 || opt.accept_p32 > (1ull << 32))
        slm::fail(SLM_ERR_INVALID_ARGUMENT, "options out of range");
    g->levels.clear();
    g->trace.clear();
    g->has_run = false;
    g->top = slm_level_stats{};
    const int32_t n0 = g->n0;
    g->final_comp.alloc(4 * (size_t)(n0 > 0 ? n0 : 1), st);
    if (n0 > 0) {
        k_iota<<<slm::grid_for(n0, 256), 256, 0, st>>>(n0, g->final_comp.as<int32_t>());
        SLM_LAUNCH_CHECK();
    }
    slm::HostCounters hc;
    for (int k = 0; k < 8; k++) { g->phase_ms[k] = 0; g->phase_cnt[k] = 0; }
    for (int k = 0; k < slm::kPosPhases; k++) g->pos_ns[k] = 0;
    for (int k = 0; k < slm::kNumBuckets; k++) g->bucket_ms[k] = 0;
    PhaseTimer tmr((opt.flags & SLM_FLAG_TIMING) != 0, st, g->phase_ms, g->phase_cnt);
    PhaseTimer *tm = tmr.on ? &tmr : nullptr;
    // current level graph
    int32_t n = n0;
    int32_t nnz = g->nnz0;
    const int32_t *rp = g->rp.as<int32_t>(), *col = g->col.as<int32_t>(), *w = g->w.as<int32_t>();
    const ST *s = NM::kDirected ? reinterpret_cast<const ST *>(g->s2.get())
                                : reinterpret_cast<const ST *>(g->s.get());
    DevBuf lrp, lcol, lw, ls;  // owned aggregated graph
    const long long m = g->m;
    Work W;
    W.ps.profile = tm != nullptr;
    g->scan_by_level.clear();
    for (int t = 0; n > 0; t++) {
        slm::check_run_control();
        const double scan_ms0 = g->phase_ms[kPhScan];
        const long long scan_cnt0 = g->phase_cnt[kPhScan];
        auto note_scans = [&] {
            g->scan_by_level.push_back({g->phase_ms[kPhScan] - scan_ms0, g->phase_cnt[kPhScan] - scan_cnt0});
        };
        if (tm) tm->start();
        W.init(n, rp, st);
        W.bk.prof_ms = (tm && t == 0) ? g->bucket_ms : nullptr;
        if (tm) tm->stop(kPhLevel);
        slm_level_stats stt{};
        stt.n = n;
        stt.nnz = nnz;
        if (tm) tm->start();
        slm::assign_nodes<NM>(n, rp, col, w, s, m, W.bk, W.a.as<int32_t>(), st);
        if (tm) tm->stop(kPhAssign);
        if (tm) tm->start();
        slm::forest_analyse(n, W.a.as<int32_t>(), W.f, st);
        if (tm) tm->stop(kPhComponents);
        if (!(opt.flags & SLM_FLAG_NO_POSITIVE)) stt.splits += positive_all<NM>(n, rp, col, w, s, m, W, st, tm);
        int sweep = 0;
        int status = 2;
        for (; sweep < opt.max_sweeps; sweep++) {
            slm::check_run_control();
            SweepCounts c = maximal_once<NM>(n, rp, col, w, s, m, W, opt.seed, opt.accept_p32, t, sweep,
                                         st, hc, tm);
            stt.candidates += c.cand;
            stt.edges_scanned += nnz;
            if (c.cand == 0) {
                status = 0;
                g->trace.push_back({t, sweep, 0, 0, 0, 0});
                sweep++;
                break;
            }
            if (c.pos == 0) {
                status = 1;
                g->trace.push_back({t, sweep, c.cand, 0, 0, 0});
                sweep++;
                break;
            }
            long long spl = 0;
            stt.moves += c.acc;
            if (c.acc > 0) {
                if (tm) tm->start();
                // names before the moves: the next POSITIVE examines only the
                // communities whose membership the moves changed
                SLM_CUDA(cudaMemcpyAsync(W.prev_root.get(), W.f.root, 4 * (size_t)n,
                                         cudaMemcpyDeviceToDevice, st));
                // only the communities the write touched change: their nodes
                // form a set closed under the new assignments
                // (many moves: the touched set is most of the graph, and the
                // full pass is cheaper than listing it)
                const int32_t na = 16LL * c.acc > n ? n : slm::moved_members(
                    n, W.acclist.as<int32_t>(), reinterpret_cast<int32_t *>(W.ctr() + 2), (int32_t)c.acc,
                    W.f.root, W.best.as<int32_t>(), W.alist.as<int32_t>(), W.amark, W.ascratch, W.atot, st);
                if (2LL * na > n) slm::forest_analyse(n, W.a.as<int32_t>(), W.f, st);
                else slm::forest_analyse_subset(na, W.alist.as<int32_t>(), W.a.as<int32_t>(), W.f, st);
                if (tm) tm->stop(kPhComponents);
                if (!(opt.flags & SLM_FLAG_NO_POSITIVE))
                    spl = positive_all<NM>(n, rp, col, w, s, m, W, st, tm, 16LL * c.acc <= n);
                stt.splits += spl;
            }
            g->trace.push_back({t, sweep, c.cand, c.pos, c.acc, spl});
        }
        stt.sweeps = sweep;
        stt.status = status;
        if (status == 2 && (opt.flags & SLM_FLAG_STRICT))
            slm::fail(SLM_ERR_NOT_CONVERGED, "sweep limit reached");
        if (tm) tm->start();
        DevBuf id(4 * (size_t)n, st), scratch(4 * (size_t)n, st);
        int32_t K = slm::compact_labels(n, W.f.root, id.as<int32_t>(), scratch.as<int32_t>(), st);
        stt.n_communities = K;
        note_scans();
        if (K == n) {
            if (tm) tm->stop(kPhLevel);
            g->top = stt;
            break;
        }
        slm::compose_labels(n0, g->final_comp.as<int32_t>(), id.as<int32_t>(), st);
        slm_graph::Level L;
        L.n = n;
        L.K = K;
        L.st = stt;
        L.comp.alloc(4 * (size_t)n0, st);
        SLM_CUDA(cudaMemcpyAsync(L.comp.get(), g->final_comp.get(), 4 * (size_t)n0,
                                 cudaMemcpyDeviceToDevice, st));
        // AGGREGATE
        DevBuf nrp, ncol, nw;
        int32_t nnz2 = slm::aggregate_graph(n, rp, col, w, id.as<int32_t>(), K, nrp, ncol, nw, st);
        // strengths of the next level: row sums of the aggregated graph, or
        // for a directed graph the (out, in) pairs summed per community
        DevBuf ns(sizeof(ST) * (size_t)(K > 0 ? K : 1), st);
        if (NM::kDirected)
            slm::sum_strengths_by(n, id.as<int32_t>(), reinterpret_cast<const unsigned long long *>(s), K,
                                  ns.as<unsigned long long>(), st);
        else
            slm::strengths(K, nrp.as<int32_t>(), nw.as<int32_t>(), ns.as<int32_t>(), st);
        L.labels = std::move(id);
        g->levels.push_back(std::move(L));
        lrp = std::move(nrp);
        lcol = std::move(ncol);
        lw = std::move(nw);
        ls = std::move(ns);
        rp = lrp.as<int32_t>();
        col = lcol.as<int32_t>();
        w = lw.as<int32_t>();
        s = ls.as<ST>();
        n = K;
        nnz = nnz2;
        if (tm) tm->stop(kPhLevel);
        if (t + 1 >= opt.max_levels) break;
    }
    slm::stream_sync(st);
    for (int k = 0; k < slm::kPosPhases; k++) g->pos_ns[k] = W.ps.prof_ns[k];
    g->has_run = true;
}

// Colour-synchronous Louvain (k_louvain.cu): per level a first-fit colouring,
// then passes over the colour classes, each class one scan of its nodes on
// the communities and totals as they stand, then its moves at once.  A level
// ends at a pass without moves (status 0), at a pass that raises the exact
// numerator by at most floor(m_w^2 / 2^20) (status 1: moves taken together
// can undo one another's gains, so passes need not settle), or at the pass
// limit (status 2); levels then compact in name order and aggregate as the
// method's do.
// colour classes of at most this many nodes may decide node by node
constexpr int32_t kLouvainDirectMaxClass = 8192;

void louvain_impl(slm_graph *g, unsigned long long seed, int max_passes, int max_levels,
                  cudaStream_t st) {
    if (g->directed) slm::fail(SLM_ERR_INVALID_ARGUMENT, "colour-synchronous Louvain takes a symmetric graph");
    if (max_passes < 1 || max_passes > 65535 || max_levels < 0 || max_levels > 65535)
        slm::fail(SLM_ERR_INVALID_ARGUMENT, "options out of range");
    g->levels.clear();
    g->trace.clear();
    g->has_run = false;
    g->top = slm_level_stats{};
    const int32_t n0 = g->n0;
    g->final_comp.alloc(4 * (size_t)(n0 > 0 ? n0 : 1), st);
    if (n0 > 0) {
        k_iota<<<slm::grid_for(n0, 256), 256, 0, st>>>(n0, g->final_comp.as<int32_t>());
        SLM_LAUNCH_CHECK();
    }
    int32_t n = n0, nnz = g->nnz0;
    const int32_t *rp = g->rp.as<int32_t>(), *col = g->col.as<int32_t>(), *w = g->w.as<int32_t>();
    const int32_t *s = g->s.as<int32_t>();
    DevBuf lrp, lcol, lw, ls;  // owned aggregated graph
    const long long m = g->m;
    DevBuf ctr(64, st), cs_all;
    unsigned long long *moves_dev = ctr.as<unsigned long long>();
    for (int t = 0; n > 0; t++) {
        slm::check_run_control();
        const size_t N = (size_t)n;
        DevBuf colour(4 * N, st), order(4 * N, st), comm(4 * N, st), sigma(4 * N, st),
            best(4 * N, st), gain(8 * N, st), kown(4 * N, st);
        const std::vector<int32_t> coff = slm::colour_nodes(n, rp, col, seed, t, colour.as<int32_t>(),
                                                            order.as<int32_t>(), st);
        const int ncol = (int)coff.size() - 1;
        // A colour class of at most kLouvainDirectMaxClass nodes whose rows
        // all have at most kLouvainDecideMaxRow entries decides node by node,
        // one block per node (two launches per class and pass); a larger class,
        // or one with longer rows (hubs), gets its own scan layout, all of them
        // on one stream and one (community, total) array.
        const std::vector<int32_t> cls_max = slm::class_max_rows(n, rp, colour.as<int32_t>(), ncol, st);
        std::vector<std::unique_ptr<slm::Buckets>> cls(ncol);
        for (int k = 0; k < ncol; k++) {
            if (coff[k + 1] - coff[k] <= kLouvainDirectMaxClass && cls_max[k] <= slm::kLouvainDecideMaxRow)
                continue;
            cls[k].reset(new slm::Buckets());
            cls[k]->one_stream = true;
            cls[k]->cs_shared = &cs_all;
            cls[k]->build_list(coff[k + 1] - coff[k], order.as<int32_t>() + coff[k], rp, st);
        }
        slm::louvain_init(n, s, comm.as<int32_t>(), sigma.as<int32_t>(), st);
        slm_level_stats stt{};
        stt.n = n;
        stt.nnz = nnz;
        int passes = 0;
        long long first_moves = 0;
        int status = 2;
        const long long theta = (long long)(((unsigned long long)m * (unsigned long long)m) >> 20);
        long long num = slm::modularity_num(n, rp, col, w, comm.as<int32_t>(), m, st);
        while (passes < max_passes) {
            slm::check_run_control();
            SLM_CUDA(cudaMemsetAsync(ctr.get(), 0, 64, st));
            for (int k = 0; k < ncol; k++) {
                if (!cls[k])
                    slm::louvain_decide(order.as<int32_t>() + coff[k], coff[k + 1] - coff[k], rp, col, w, s, m,
                                        comm.as<int32_t>(), sigma.as<int32_t>(), cls_max[k], best.as<int32_t>(), st);
                else
                    slm::scan_nodes<slm::NMSym>(n, rp, col, w, s, m, comm.as<int32_t>(), sigma.as<int32_t>(),
                                                *cls[k], best.as<int32_t>(), gain.as<long long>(),
                                                kown.as<int32_t>(), moves_dev + 1, st);
                slm::louvain_move(order.as<int32_t>() + coff[k], coff[k + 1] - coff[k], best.as<int32_t>(),
                                  comm.as<int32_t>(), s, sigma.as<int32_t>(), moves_dev, st);
            }
            unsigned long long mv = 0;
            SLM_CUDA(cudaMemcpyAsync(&mv, moves_dev, sizeof mv, cudaMemcpyDeviceToHost, st));
            slm::stream_sync(st);
            g->trace.push_back({t, passes, 0, 0, (long long)mv, 0});
            passes++;
            stt.moves += (long long)mv;
            stt.edges_scanned += nnz;
            if (passes == 1) first_moves = (long long)mv;
            if (mv == 0) {
                status = 0;
                break;
            }
            const long long num2 = slm::modularity_num(n, rp, col, w, comm.as<int32_t>(), m, st);
            const long long gain = num2 - num;
            num = num2;
            if (gain <= theta) {
                status = 1;
                break;
            }
        }
        stt.sweeps = passes;
        stt.status = status;
        DevBuf id(4 * N, st), scratch(4 * N, st);
        const int32_t K = slm::compact_names(n, comm.as<int32_t>(), id.as<int32_t>(), scratch.as<int32_t>(), st);
        stt.n_communities = K;
        if (first_moves == 0 || K == n) {
            g->top = stt;
            break;
        }
        slm::compose_labels(n0, g->final_comp.as<int32_t>(), id.as<int32_t>(), st);
        slm_graph::Level L;
        L.n = n;
        L.K = K;
        L.st = stt;
        L.comp.alloc(4 * (size_t)n0, st);
        SLM_CUDA(cudaMemcpyAsync(L.comp.get(), g->final_comp.get(), 4 * (size_t)n0,
                                 cudaMemcpyDeviceToDevice, st));
        DevBuf nrp, ncol_, nw;
        const int32_t nnz2 = slm::aggregate_graph(n, rp, col, w, id.as<int32_t>(), K, nrp, ncol_, nw, st);
        DevBuf ns(4 * (size_t)(K > 0 ? K : 1), st);
        slm::strengths(K, nrp.as<int32_t>(), nw.as<int32_t>(), ns.as<int32_t>(), st);
        L.labels = std::move(id);
        g->levels.push_back(std::move(L));
        lrp = std::move(nrp);
        lcol = std::move(ncol_);
        lw = std::move(nw);
        ls = std::move(ns);
        rp = lrp.as<int32_t>();
        col = lcol.as<int32_t>();
        w = lw.as<int32_t>();
        s = ls.as<int32_t>();
        n = K;
        nnz = nnz2;
        if (t + 1 >= max_levels) break;
    }
    slm::stream_sync(st);
    g->has_run = true;
}

void check_csr_host(int32_t n, const int32_t *rp_h, long long *nnz) {
    if (rp_h[0] != 0) slm::fail(SLM_ERR_INVALID_ARGUMENT, "row_ptr[0] must be 0");
    for (int32_t i = 0; i < n; i++)
        if (rp_h[i + 1] < rp_h[i]) slm::fail(SLM_ERR_INVALID_ARGUMENT, "row_ptr must be non-decreasing");
    *nnz = rp_h[n];
}

}  // namespace

extern "C" {

void slm_default_options(slm_options *opt) {
    if (!opt) return;
    opt->seed = 1;
    opt->accept_p32 = 1ull << 31;
    opt->max_sweeps = 1000;
    opt->max_levels = 64;
    opt->flags = 0;
}

const char *slm_status_string(slm_status s) {
    switch (s) {
    case SLM_OK: return "ok";
    case SLM_ERR_INVALID_ARGUMENT: return "invalid argument";
    case SLM_ERR_NOT_SYMMETRIC: return "matrix not symmetric";
    case SLM_ERR_OVERFLOW: return "total weight must be below 2^31";
    case SLM_ERR_OUT_OF_MEMORY: return "out of device memory";
    case SLM_ERR_CUDA: return "CUDA error";
    case SLM_ERR_NOT_RUN: return "slm_run has not completed on this graph";
    case SLM_ERR_NOT_CONVERGED: return "sweep limit reached";
    case SLM_ERR_TIMEOUT: return "timeout";
    case SLM_ERR_BUDGET: return "memory budget exceeded";
    case SLM_ERR_CANCELLED: return "request cancelled";
    case SLM_ERR_DEADLINE: return "request deadline passed";
    }
    return "unknown status";
}

const char *slm_last_error(const slm_graph *g) {
    return g ? g->err.c_str() : g_create_error.c_str();
}

slm_status slm_create_graph(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                            const int32_t *weights, int where, void *stream, slm_graph **out) {
    if (!out) return SLM_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    auto g = std::make_unique<slm_graph>();
    slm_status st = guarded(nullptr, [&] {
        cudaStream_t s = as_stream(stream);
        if (n < 0 || !row_ptr || (where != SLM_HOST && where != SLM_DEVICE))
            slm::fail(SLM_ERR_INVALID_ARGUMENT, "bad n, row_ptr or where");
        std::vector<int32_t> rp_h((size_t)n + 1);
        cudaMemcpyKind kind = where == SLM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
        if (where == SLM_HOST) std::memcpy(rp_h.data(), row_ptr, sizeof(int32_t) * rp_h.size());
        else {
            SLM_CUDA(cudaMemcpyAsync(rp_h.data(), row_ptr, sizeof(int32_t) * rp_h.size(),
                                     cudaMemcpyDeviceToHost, s));
            slm::stream_sync(s);
        }
        long long nnz = 0;
        check_csr_host(n, rp_h.data(), &nnz);
        if (nnz >= (1LL << 31)) slm::fail(SLM_ERR_OVERFLOW, "too many entries");
        if (nnz > 0 && !col_idx) slm::fail(SLM_ERR_INVALID_ARGUMENT, "col_idx is NULL");
        g->n0 = n;
        g->nnz0 = (int32_t)nnz;
        g->rp.alloc(4 * ((size_t)n + 1), s);
        g->col.alloc(4 * (size_t)(nnz > 0 ? nnz : 1), s);
        g->w.alloc(4 * (size_t)(nnz > 0 ? nnz : 1), s);
        g->s.alloc(4 * (size_t)(n > 0 ? n : 1), s);
        SLM_CUDA(cudaMemcpyAsync(g->rp.get(), rp_h.data(), 4 * ((size_t)n + 1),
                                 cudaMemcpyHostToDevice, s));
        if (nnz > 0) {
            SLM_CUDA(cudaMemcpyAsync(g->col.get(), col_idx, 4 * (size_t)nnz, kind, s));
            if (weights) SLM_CUDA(cudaMemcpyAsync(g->w.get(), weights, 4 * (size_t)nnz, kind, s));
            else {
                k_fill_ones<<<slm::grid_for(nnz, 256), 256, 0, s>>>(nnz, g->w.as<int32_t>());
                SLM_LAUNCH_CHECK();
            }
        }
        int bad = slm::validate_csr(n, nnz, g->rp.as<int32_t>(), g->col.as<int32_t>(), g->w.as<int32_t>(), s);
        if (bad & (1 | 8)) slm::fail(SLM_ERR_INVALID_ARGUMENT, "column index out of range, unsorted or duplicated");
        if (bad & 2) slm::fail(SLM_ERR_INVALID_ARGUMENT, "non-positive weight");
        if (bad & 4) slm::fail(SLM_ERR_NOT_SYMMETRIC, "W is not symmetric");
        // m_w < 2^31 keeps every gain exact in int64; the weights sum is
        // bounded first so that the per-node strengths fit in int32
        g->m = slm::strengths(n, g->rp.as<int32_t>(), g->w.as<int32_t>(), g->s.as<int32_t>(), s);
        if (g->m >= (1LL << 31)) slm::fail(SLM_ERR_OVERFLOW, "m_w must be below 2^31");
        slm::stream_sync(s);
    });
    if (st == SLM_OK) *out = g.release();
    return st;
}

slm_status slm_create_graph_directed(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                                     const int32_t *weights, int where, void *stream,
                                     slm_graph **out) {
    if (!out) return SLM_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    auto g = std::make_unique<slm_graph>();
    slm_status st = guarded(nullptr, [&] {
        cudaStream_t s = as_stream(stream);
        if (n < 0 || !row_ptr || (where != SLM_HOST && where != SLM_DEVICE))
            slm::fail(SLM_ERR_INVALID_ARGUMENT, "bad n, row_ptr or where");
        // W on the host: U = W + W^T is built here, once
        std::vector<int32_t> rp((size_t)n + 1);
        auto fetch = [&](void *dst, const void *src, size_t bytes) {
            if (where == SLM_HOST) std::memcpy(dst, src, bytes);
            else SLM_CUDA(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
        };
        fetch(rp.data(), row_ptr, sizeof(int32_t) * rp.size());
        long long nnz = 0;
        check_csr_host(n, rp.data(), &nnz);
        if (nnz >= (1LL << 30)) slm::fail(SLM_ERR_OVERFLOW, "too many entries");
        if (nnz > 0 && !col_idx) slm::fail(SLM_ERR_INVALID_ARGUMENT, "col_idx is NULL");
        std::vector<int32_t> col((size_t)nnz), w((size_t)nnz, 1);
        if (nnz > 0) {
            fetch(col.data(), col_idx, sizeof(int32_t) * (size_t)nnz);
            if (weights) fetch(w.data(), weights, sizeof(int32_t) * (size_t)nnz);
        }
        std::vector<long long> so((size_t)n, 0), si((size_t)n, 0);
        long long m = 0;
        for (int32_t i = 0; i < n; i++)
            for (int32_t p = rp[i]; p < rp[i + 1]; p++) {
                const int32_t j = col[p];
                if (j < 0 || j >= n || (p > rp[i] && j <= col[p - 1]))
                    slm::fail(SLM_ERR_INVALID_ARGUMENT, "column index out of range, unsorted or duplicated");
                if (w[p] <= 0) slm::fail(SLM_ERR_INVALID_ARGUMENT, "non-positive weight");
                so[i] += w[p];
                si[j] += w[p];
                m += w[p];
                // m_w < 2^30 keeps every packed total and every int64 gain exact
                if (m >= (1LL << 30)) slm::fail(SLM_ERR_OVERFLOW, "m_w must be below 2^30 for a directed graph");
            }
        // W^T by counting (its rows come out with ascending columns), then
        // row i of U merges row i of W and row i of W^T
        std::vector<int32_t> tp((size_t)n + 1, 0), tc((size_t)nnz), tw((size_t)nnz);
        for (long long p = 0; p < nnz; p++) tp[(size_t)col[p] + 1]++;
        for (int32_t v = 0; v < n; v++) tp[v + 1] += tp[v];
        std::vector<int32_t> fill(tp.begin(), tp.end() - 1);
        for (int32_t i = 0; i < n; i++)
            for (int32_t p = rp[i]; p < rp[i + 1]; p++) {
                const int32_t q = fill[col[p]]++;
                tc[q] = i;
                tw[q] = w[p];
            }
        std::vector<int32_t> urp((size_t)n + 1, 0), ucol, uw;
        ucol.reserve((size_t)(2 * nnz));
        uw.reserve((size_t)(2 * nnz));
        for (int32_t i = 0; i < n; i++) {
            int32_t x = rp[i], y = tp[i];
            while (x < rp[i + 1] || y < tp[i + 1]) {
                if (y >= tp[i + 1] || (x < rp[i + 1] && col[x] < tc[y])) {
                    ucol.push_back(col[x]); uw.push_back(w[x]); x++;
                } else if (x >= rp[i + 1] || tc[y] < col[x]) {
                    ucol.push_back(tc[y]); uw.push_back(tw[y]); y++;
                } else {
                    ucol.push_back(col[x]); uw.push_back(w[x] + tw[y]); x++; y++;
                }
            }
            urp[i + 1] = (int32_t)ucol.size();
        }
        const long long nnzu = (long long)ucol.size();
        std::vector<unsigned long long> s2((size_t)n);
        for (int32_t i = 0; i < n; i++) s2[i] = ((unsigned long long)so[i] << 32) | (unsigned long long)si[i];
        g->directed = true;
        g->n0 = n;
        g->nnz0 = (int32_t)nnzu;
        g->m = m;
        g->rp.alloc(4 * ((size_t)n + 1), s);
        g->col.alloc(4 * (size_t)(nnzu > 0 ? nnzu : 1), s);
        g->w.alloc(4 * (size_t)(nnzu > 0 ? nnzu : 1), s);
        g->s.alloc(16, s);
        g->s2.alloc(8 * (size_t)(n > 0 ? n : 1), s);
        SLM_CUDA(cudaMemcpyAsync(g->rp.get(), urp.data(), 4 * ((size_t)n + 1), cudaMemcpyHostToDevice, s));
        if (nnzu > 0) {
            SLM_CUDA(cudaMemcpyAsync(g->col.get(), ucol.data(), 4 * (size_t)nnzu, cudaMemcpyHostToDevice, s));
            SLM_CUDA(cudaMemcpyAsync(g->w.get(), uw.data(), 4 * (size_t)nnzu, cudaMemcpyHostToDevice, s));
        }
        if (n > 0)
            SLM_CUDA(cudaMemcpyAsync(g->s2.get(), s2.data(), 8 * (size_t)n, cudaMemcpyHostToDevice, s));
        slm::stream_sync(s);  // the host vectors go out of scope
    });
    if (st == SLM_OK) *out = g.release();
    return st;
}

int32_t slm_graph_is_directed(const slm_graph *g) { return g && g->directed ? 1 : 0; }

slm_status slm_run(slm_graph *g, const slm_options *opt, void *stream) {
    if (!g) return SLM_ERR_INVALID_ARGUMENT;
    slm_options o;
    slm_default_options(&o);
    if (opt) o = *opt;
    // the previous run's results, put back when this run fails
    std::vector<slm_graph::Level> levels = std::move(g->levels);
    std::vector<std::array<long long, 6>> trace = std::move(g->trace);
    const slm_level_stats top = g->top;
    DevBuf comp = std::move(g->final_comp);
    const bool had_run = g->has_run;
    g->levels.clear();
    g->trace.clear();
    const slm_status st = guarded(g, [&] {
        if (g->directed) run_impl<slm::NMDir>(g, o, as_stream(stream));
        else run_impl<slm::NMSym>(g, o, as_stream(stream));
    });
    if (st != SLM_OK) {
        g->levels = std::move(levels);
        g->trace = std::move(trace);
        g->top = top;
        g->final_comp = std::move(comp);
        g->has_run = had_run;
    }
    return st;
}

slm_status slm_run_louvain(slm_graph *g, uint64_t seed, int32_t max_passes, int32_t max_levels,
                           void *stream) {
    if (!g) return SLM_ERR_INVALID_ARGUMENT;
    std::vector<slm_graph::Level> levels = std::move(g->levels);
    std::vector<std::array<long long, 6>> trace = std::move(g->trace);
    const slm_level_stats top = g->top;
    DevBuf comp = std::move(g->final_comp);
    const bool had_run = g->has_run;
    g->levels.clear();
    g->trace.clear();
    const slm_status st = guarded(g, [&] { louvain_impl(g, seed, max_passes, max_levels, as_stream(stream)); });
    if (st != SLM_OK) {
        g->levels = std::move(levels);
        g->trace = std::move(trace);
        g->top = top;
        g->final_comp = std::move(comp);
        g->has_run = had_run;
    }
    return st;
}

slm_status slm_num_levels(const slm_graph *g, int32_t *levels) {
    if (!g || !levels) return SLM_ERR_INVALID_ARGUMENT;
    if (!g->has_run) return SLM_ERR_NOT_RUN;
    *levels = (int32_t)g->levels.size();
    return SLM_OK;
}

slm_status slm_get_partition(const slm_graph *g, int32_t level, int32_t *labels, int where,
                             int32_t *n_communities) {
    if (!g) return SLM_ERR_INVALID_ARGUMENT;
    if (!g->has_run) return SLM_ERR_NOT_RUN;
    if (level < -1 || level >= (int32_t)g->levels.size()) return SLM_ERR_INVALID_ARGUMENT;
    if (where != SLM_HOST && where != SLM_DEVICE) return SLM_ERR_INVALID_ARGUMENT;
    slm_graph *gm = const_cast<slm_graph *>(g);
    return guarded(gm, [&] {
        const DevBuf *src;
        size_t count;
        int32_t K;
        if (level == -1) {
            src = &g->final_comp;
            count = (size_t)g->n0;
            K = g->levels.empty() ? g->n0 : g->levels.back().K;
        } else {
            src = &g->levels[level].labels;
            count = (size_t)g->levels[level].n;
            K = g->levels[level].K;
        }
        if (count > 0) {
            if (!labels) slm::fail(SLM_ERR_INVALID_ARGUMENT, "labels is NULL");
            SLM_CUDA(cudaMemcpy(labels, src->get(), 4 * count,
                                where == SLM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice));
        }
        if (n_communities) *n_communities = K;
    });
}

}  // extern "C"

namespace {
// exact numerator of a labelling of the input nodes, for either kind of graph
long long graph_modularity_num(const slm_graph *g, const int32_t *labels) {
    if (g->directed)
        return slm::modularity_num_directed(g->n0, g->rp.as<int32_t>(), g->col.as<int32_t>(),
                                            g->w.as<int32_t>(), g->s2.as<unsigned long long>(),
                                            labels, g->m, nullptr);
    return slm::modularity_num(g->n0, g->rp.as<int32_t>(), g->col.as<int32_t>(),
                               g->w.as<int32_t>(), labels, g->m, nullptr);
}
}  // namespace

extern "C" {

slm_status slm_modularity(const slm_graph *g, int32_t level, double *q) {
    if (!g || !q) return SLM_ERR_INVALID_ARGUMENT;
    if (!g->has_run) return SLM_ERR_NOT_RUN;
    if (level < -1 || level >= (int32_t)g->levels.size()) return SLM_ERR_INVALID_ARGUMENT;
    slm_graph *gm = const_cast<slm_graph *>(g);
    return guarded(gm, [&] {
        const DevBuf &lab = level == -1 ? g->final_comp : g->levels[level].comp;
        long long num = graph_modularity_num(g, lab.as<int32_t>());
        *q = slm::modularity_from_num(num, g->m);
    });
}

slm_status slm_modularity_of(const slm_graph *g, const int32_t *labels, int where, double *q) {
    if (!g || !q || (g->n0 > 0 && !labels)) return SLM_ERR_INVALID_ARGUMENT;
    if (where != SLM_HOST && where != SLM_DEVICE) return SLM_ERR_INVALID_ARGUMENT;
    slm_graph *gm = const_cast<slm_graph *>(g);
    return guarded(gm, [&] {
        DevBuf lab(4 * (size_t)(g->n0 > 0 ? g->n0 : 1), nullptr);
        if (g->n0 > 0)
            SLM_CUDA(cudaMemcpy(lab.get(), labels, 4 * (size_t)g->n0,
                                where == SLM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice));
        // labels must name nodes of the graph
        std::vector<int32_t> h((size_t)g->n0);
        if (g->n0 > 0) SLM_CUDA(cudaMemcpy(h.data(), lab.get(), 4 * h.size(), cudaMemcpyDeviceToHost));
        for (int32_t v : h)
            if (v < 0 || v >= g->n0) slm::fail(SLM_ERR_INVALID_ARGUMENT, "label out of range");
        long long num = graph_modularity_num(g, lab.as<int32_t>());
        *q = slm::modularity_from_num(num, g->m);
    });
}

slm_status slm_get_stats(const slm_graph *g, int32_t level, slm_level_stats *st) {
    if (!g || !st) return SLM_ERR_INVALID_ARGUMENT;
    if (!g->has_run) return SLM_ERR_NOT_RUN;
    if (level < -1 || level >= (int32_t)g->levels.size()) return SLM_ERR_INVALID_ARGUMENT;
    *st = level == -1 ? g->top : g->levels[level].st;
    return SLM_OK;
}

slm_status slm_get_trace(const slm_graph *g, int64_t *rows, int64_t cap, int64_t *len) {
    if (!g || !len) return SLM_ERR_INVALID_ARGUMENT;
    *len = (int64_t)g->trace.size();
    for (int64_t r = 0; r < cap && r < *len; r++)
        for (int k = 0; k < 6; k++) rows[6 * r + k] = g->trace[r][k];
    return SLM_OK;
}

slm_status slm_get_timing(const slm_graph *g, double *ms8, int64_t *count8) {
    if (!g || !ms8 || !count8) return SLM_ERR_INVALID_ARGUMENT;
    for (int k = 0; k < 8; k++) {
        ms8[k] = g->phase_ms[k];
        count8[k] = g->phase_cnt[k];
    }
    return SLM_OK;
}

slm_status slm_get_scan_timing(const slm_graph *g, int32_t level, double *ms, int64_t *count) {
    if (!g || !ms || !count) return SLM_ERR_INVALID_ARGUMENT;
    if (!g->has_run) return SLM_ERR_NOT_RUN;
    const int32_t L = (int32_t)g->levels.size();
    if (level < -1 || level >= L) return SLM_ERR_INVALID_ARGUMENT;
    const size_t k = level == -1 ? (size_t)L : (size_t)level;
    if (k >= g->scan_by_level.size()) {
        *ms = 0;
        *count = 0;
        return SLM_OK;
    }
    *ms = g->scan_by_level[k].first;
    *count = g->scan_by_level[k].second;
    return SLM_OK;
}

slm_status slm_set_scan_tuning(const slm_scan_tuning *t) {
    if (!t || (t->streams != 1 && t->streams != 4)) return SLM_ERR_INVALID_ARGUMENT;
    for (int32_t v : {t->blocks_large, t->blocks_mid, t->blocks_small, t->blocks_warp,
                      t->blocks_hub, t->blocks_group})
        if (v < 1 || v > 64) return SLM_ERR_INVALID_ARGUMENT;
    if (t->shape_alt < 0 || t->shape_alt >= (1 << 11)) return SLM_ERR_INVALID_ARGUMENT;
    slm::ScanTuning u;
    u.streams = t->streams;
    u.blocks_large = t->blocks_large;
    u.blocks_mid = t->blocks_mid;
    u.blocks_small = t->blocks_small;
    u.blocks_warp = t->blocks_warp;
    u.blocks_hub = t->blocks_hub;
    u.blocks_group = t->blocks_group;
    u.shape_alt = t->shape_alt;
    slm::set_scan_tuning(u);
    return SLM_OK;
}

slm_status slm_get_scan_tuning(slm_scan_tuning *t) {
    if (!t) return SLM_ERR_INVALID_ARGUMENT;
    const slm::ScanTuning u = slm::scan_tuning();
    *t = slm_scan_tuning{u.streams, u.blocks_large, u.blocks_mid, u.blocks_small,
                         u.blocks_warp, u.blocks_hub, u.blocks_group, u.shape_alt};
    return SLM_OK;
}

slm_status slm_get_scan_bucket_timing(const slm_graph *g, double *ms, int32_t cap, int32_t *len) {
    if (!g || !len || cap < 0 || (cap > 0 && !ms)) return SLM_ERR_INVALID_ARGUMENT;
    *len = slm::kNumBuckets;
    for (int k = 0; k < cap && k < slm::kNumBuckets; k++) ms[k] = g->bucket_ms[k];
    return SLM_OK;
}

slm_status slm_get_positive_profile(const slm_graph *g, int64_t *ns, int32_t cap, int32_t *len) {
    if (!g || !len || cap < 0 || (cap > 0 && !ns)) return SLM_ERR_INVALID_ARGUMENT;
    *len = slm::kPosPhases;
    for (int k = 0; k < cap && k < slm::kPosPhases; k++) ns[k] = g->pos_ns[k];
    return SLM_OK;
}

uint64_t slm_launch_count(void) { return slm::launch_count(); }

void slm_debug_fail_allocation(int64_t k) { slm::set_alloc_failure(k); }

void slm_release_cached_memory(void) { slm::trim_pool(); }

slm_status slm_check_grid_barrier(int32_t blocks, int32_t absent_block, double limit_s,
                                  void *stream) {
    if (blocks < 1 || absent_block < -1 || absent_block >= blocks || !(limit_s > 0) || limit_s > 60)
        return SLM_ERR_INVALID_ARGUMENT;
    bool ok = false;
    slm_status st = guarded(nullptr, [&] {
        ok = slm::barrier_check(blocks, absent_block, (long long)(limit_s * 1e9), as_stream(stream));
    });
    if (st != SLM_OK) return st;
    if (!ok) {
        slm::set_global_error("a grid barrier wait ran out of time");
        return SLM_ERR_TIMEOUT;
    }
    return SLM_OK;
}

void slm_destroy_graph(slm_graph *g) {
    if (!g) return;
    slm::ReleaseOnDefaultStream on_default;
    delete g;
}

// ---------------------------------------------------------------------------
// Step entry points (slm_steps.h)
// ---------------------------------------------------------------------------
#define STEP_CHECK(cond) \
    if (!(cond)) return SLM_ERR_INVALID_ARGUMENT

slm_status slm_step_strengths(int32_t n, const int32_t *row_ptr, const int32_t *col,
                              const int32_t *w, int32_t *s, int64_t *m_w_host, void *stream) {
    STEP_CHECK(n >= 0 && (n == 0 || (row_ptr && w && s)) && m_w_host);
    (void)col;
    return guarded(nullptr, [&] {
        *m_w_host = slm::strengths(n, row_ptr, w, s, as_stream(stream));
    });
}

slm_status slm_step_assign(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *w,
                           const int32_t *s, int64_t m_w, int32_t *a, void *stream) {
    STEP_CHECK(n >= 0 && (n == 0 || (row_ptr && col && w && s && a)));
    return guarded(nullptr, [&] {
        cudaStream_t st = as_stream(stream);
        slm::Buckets bk;
        bk.build(n, row_ptr, st);
        slm::assign_nodes<slm::NMSym>(n, row_ptr, col, w, s, m_w, bk, a, st);
        slm::stream_sync(st);
    });
}

slm_status slm_step_components(int32_t n, const int32_t *a, int32_t *root, void *stream) {
    STEP_CHECK(n >= 0 && (n == 0 || (a && root)));
    return guarded(nullptr, [&] {
        cudaStream_t st = as_stream(stream);
        if (slm::count_out_of_range(n, a, n, st)) slm::fail(SLM_ERR_INVALID_ARGUMENT, "a[v] outside [0, n)");
        size_t N = (size_t)(n > 0 ? n : 1);
        DevBuf oc(N, st), en(4 * N, st), de(4 * N, st), cd(4 * N, st), ja(8 * N, st), jb(8 * N, st);
        slm::Forest f;
        f.root = root;
        f.oncycle = oc.as<uint8_t>();
        f.entry = en.as<int32_t>();
        f.depth = de.as<int32_t>();
        f.cdist = cd.as<int32_t>();
        f.jmpA = ja.as<int2>();
        f.jmpB = jb.as<int2>();
        slm::forest_analyse(n, a, f, st);
        slm::stream_sync(st);
    });
}

namespace {
// A level workspace whose assignment and forest describe the caller's state.
void load_state(Work &W, int32_t n, const int32_t *rp, const int32_t *a, cudaStream_t st) {
    if (slm::count_out_of_range(n, a, n, st)) slm::fail(SLM_ERR_INVALID_ARGUMENT, "a[v] outside [0, n)");
    W.init(n, rp, st);
    if (n > 0)
        SLM_CUDA(cudaMemcpyAsync(W.a.get(), a, 4 * (size_t)n, cudaMemcpyDeviceToDevice, st));
    slm::forest_analyse(n, W.a.as<int32_t>(), W.f, st);
}
}  // namespace

slm_status slm_step_scan(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *w,
                         const int32_t *s, int64_t m_w, const int32_t *root, int32_t *best,
                         int64_t *gain, int64_t *g_out, void *stream) {
    STEP_CHECK(n >= 0 && (n == 0 || (row_ptr && col && w && s && root && best && gain)));
    return guarded(nullptr, [&] {
        cudaStream_t st = as_stream(stream);
        if (slm::count_out_of_range(n, root, n, st)) slm::fail(SLM_ERR_INVALID_ARGUMENT, "root[v] outside [0, n)");
        Work W;
        W.init(n, row_ptr, st);
        slm::community_sigma(n, root, s, W.sigma.as<int32_t>(), st);
        SLM_CUDA(cudaMemsetAsync(W.ctr(), 0, 64, st));
        slm::scan_nodes<slm::NMSym>(n, row_ptr, col, w, s, m_w, root, W.sigma.as<int32_t>(), W.bk, best,
                        reinterpret_cast<long long *>(gain), W.kown.as<int32_t>(), W.ctr(), st);
        if (g_out && n > 0) {
            // own-community weights without the scan's early outs, then g
            DevBuf flag(4 * (size_t)n, st);
            SLM_CUDA(cudaMemsetAsync(flag.get(), 0, 4 * (size_t)n, st));
            slm::own_weight_nodes<slm::NMSym>(n, row_ptr, col, w, s, m_w, root, W.sigma.as<int32_t>(), W.bk,
                                  W.kown.as<int32_t>(), flag.as<int32_t>(), st);
            slm::local_gain_nodes<slm::NMSym>(n, s, m_w, root, W.sigma.as<int32_t>(), W.kown.as<int32_t>(),
                                  reinterpret_cast<long long *>(g_out), st);
        }
        slm::stream_sync(st);
    });
}

slm_status slm_step_branch_gain(int32_t n, const int32_t *row_ptr, const int32_t *col,
                                const int32_t *w, const int32_t *s, int64_t m_w, const int32_t *a,
                                const int32_t *root, const int32_t *best, const int64_t *gain,
                                int64_t *bg, void *stream) {
    STEP_CHECK(n >= 0 && (n == 0 || (row_ptr && col && w && s && a && root && best && gain && bg)));
    (void)root;
    return guarded(nullptr, [&] {
        cudaStream_t st = as_stream(stream);
        Work W;
        load_state(W, n, row_ptr, a, st);
        slm::community_sigma(n, W.f.root, s, W.sigma.as<int32_t>(), st);
        // own-community weights of the snapshot
        SLM_CUDA(cudaMemsetAsync(W.ctr(), 0, 64, st));
        slm::scan_nodes<slm::NMSym>(n, row_ptr, col, w, s, m_w, W.f.root, W.sigma.as<int32_t>(), W.bk,
                        W.best.as<int32_t>(), W.gain.as<long long>(), W.kown.as<int32_t>(), W.ctr(), st);
        slm::branch_gains<slm::NMSym>(n, row_ptr, col, w, s, m_w, W.a.as<int32_t>(), W.f, W.sigma.as<int32_t>(),
                          best, reinterpret_cast<const long long *>(gain), W.kown.as<int32_t>(), W.bs,
                          reinterpret_cast<long long *>(bg), st);
        slm::stream_sync(st);
    });
}

slm_status slm_step_maximal(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *w,
                            const int32_t *s, int64_t m_w, int32_t *a, const int32_t *root,
                            uint64_t seed, uint64_t accept_p32, int32_t level, int32_t sweep,
                            int64_t *counts_host, void *stream) {
    STEP_CHECK(n >= 0 && (n == 0 || (row_ptr && col && w && s && a && root)) && counts_host);
    (void)root;
    return guarded(nullptr, [&] {
        cudaStream_t st = as_stream(stream);
        Work W;
        load_state(W, n, row_ptr, a, st);
        slm::HostCounters hc;
        SweepCounts c = maximal_once<slm::NMSym>(n, row_ptr, col, w, s, m_w, W, seed, accept_p32, level, sweep,
                                     st, hc);
        if (n > 0) SLM_CUDA(cudaMemcpyAsync(a, W.a.get(), 4 * (size_t)n, cudaMemcpyDeviceToDevice, st));
        slm::stream_sync(st);
        counts_host[0] = c.cand;
        counts_host[1] = c.pos;
        counts_host[2] = c.acc;
    });
}

slm_status slm_step_positive(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *w,
                             const int32_t *s, int64_t m_w, int32_t *a, int32_t *root,
                             int64_t *splits_host, void *stream) {
    STEP_CHECK(n >= 0 && (n == 0 || (row_ptr && col && w && s && a && root)) && splits_host);
    return guarded(nullptr, [&] {
        cudaStream_t st = as_stream(stream);
        Work W;
        load_state(W, n, row_ptr, a, st);
        *splits_host = positive_all<slm::NMSym>(n, row_ptr, col, w, s, m_w, W, st);
        if (n > 0) {
            SLM_CUDA(cudaMemcpyAsync(a, W.a.get(), 4 * (size_t)n, cudaMemcpyDeviceToDevice, st));
            SLM_CUDA(cudaMemcpyAsync(root, W.f.root, 4 * (size_t)n, cudaMemcpyDeviceToDevice, st));
        }
        slm::stream_sync(st);
    });
}

slm_status slm_step_compact(int32_t n, const int32_t *root, int32_t *id, int32_t *K_host,
                            void *stream) {
    STEP_CHECK(n >= 0 && (n == 0 || (root && id)) && K_host);
    return guarded(nullptr, [&] {
        cudaStream_t st = as_stream(stream);
        DevBuf scratch(4 * (size_t)(n > 0 ? n : 1), st);
        *K_host = slm::compact_labels(n, root, id, scratch.as<int32_t>(), st);
    });
}

slm_status slm_step_aggregate(int32_t n, const int32_t *row_ptr, const int32_t *col,
                              const int32_t *w, const int32_t *id, int32_t K,
                              int32_t *row_ptr_out, int32_t *col_out, int32_t *w_out,
                              int32_t *nnz_out_host, void *stream) {
    STEP_CHECK(n >= 0 && K >= 0 && K <= (n > 0 ? n : 0) && (n == 0 || (row_ptr && col && w && id)) &&
               row_ptr_out && nnz_out_host);
    return guarded(nullptr, [&] {
        cudaStream_t st = as_stream(stream);
        DevBuf rp2, col2, w2;
        int32_t nnz2 = slm::aggregate_graph(n, row_ptr, col, w, id, K, rp2, col2, w2, st);
        SLM_CUDA(cudaMemcpyAsync(row_ptr_out, rp2.get(), 4 * ((size_t)K + 1), cudaMemcpyDeviceToDevice, st));
        if (nnz2 > 0) {
            SLM_CUDA(cudaMemcpyAsync(col_out, col2.get(), 4 * (size_t)nnz2, cudaMemcpyDeviceToDevice, st));
            SLM_CUDA(cudaMemcpyAsync(w_out, w2.get(), 4 * (size_t)nnz2, cudaMemcpyDeviceToDevice, st));
        }
        slm::stream_sync(st);
        *nnz_out_host = nnz2;
    });
}

slm_status slm_step_modularity(int32_t n, const int32_t *row_ptr, const int32_t *col,
                               const int32_t *w, const int32_t *labels, double *q_host,
                               int64_t *num_host, void *stream) {
    STEP_CHECK(n >= 0 && (n == 0 || (row_ptr && col && w && labels)) && q_host && num_host);
    return guarded(nullptr, [&] {
        cudaStream_t st = as_stream(stream);
        DevBuf s(4 * (size_t)(n > 0 ? n : 1), st);
        long long m = slm::strengths(n, row_ptr, w, s.as<int32_t>(), st);
        long long num = slm::modularity_num(n, row_ptr, col, w, labels, m, st);
        *num_host = num;
        *q_host = slm::modularity_from_num(num, m);
    });
}

}  // extern "C"
