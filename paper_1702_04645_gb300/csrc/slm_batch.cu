// slm_batch.cu -- Algorithm 1 on a forest of independent graphs (slm_batch.h).
//
// The forest is one block-diagonal CSR, so every kernel of the single-graph
// path applies to it unchanged except where m_w or the acceptance draw enter:
// those read the node's graph (MParam, RngParam).  The host keeps, per graph,
// whether it still runs at this level and its statistics; the sweep loop
// stops a graph exactly where slm_run would (no candidate, no positive branch
// gain, sweep limit), and a level ends for the batch when every graph has
// stopped.  A graph whose level finds no structure (K = n) is finished: its
// rows are dropped from the next aggregated forest, where its nodes stay as
// isolated singletons that never move.
#include <algorithm>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "driver.cuh"
#include "slm_batch.h"

using slm::DevBuf;

struct slm_batch {
    int32_t G = 0, N0 = 0, nnz0 = 0;
    std::vector<int32_t> goff0;            // host, G+1
    std::vector<unsigned long long> seeds; // host, G (empty: use opt.seed)
    std::vector<long long> mg;             // host, G
    DevBuf goff0_d, rp, col, w, s, gid0, mg_d;
    bool has_run = false;
    struct GLevel {
        int32_t n = 0, K = 0;
        slm_level_stats st{};
    };
    std::vector<std::vector<GLevel>> glev;  // per graph: recorded levels
    std::vector<slm_level_stats> gtop;      // per graph: last, unrecorded level
    std::vector<DevBuf> lev_ids;            // per batch level: ids of that level's forest
    std::vector<std::vector<int32_t>> lev_goff, lev_koff;  // node and id offsets per graph
    DevBuf final_comp;                       // composed ids of the input nodes
    std::vector<int32_t> final_koff;         // id offsets per graph of final_comp
    std::vector<double> q;                   // per graph final modularity
    int32_t batch_levels = 0;
    long long batch_sweeps = 0;
    std::string err;
};

namespace {

thread_local std::string g_batch_create_error;

template <class F> slm_status guarded_b(slm_batch *b, F &&f) {
    try {
        f();
        return SLM_OK;
    } catch (const slm::Error &e) {
        if (b) b->err = e.msg;
        else g_batch_create_error = e.msg;
        return e.status;
    } catch (const std::exception &e) {
        if (b) b->err = e.what();
        else g_batch_create_error = e.what();
        return SLM_ERR_CUDA;
    }
}

__global__ void k_iota_b(int32_t n, int32_t *p) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = (int32_t)i;
}
__global__ void k_ones_b(long long n, int32_t *p) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = 1;
}
// rp[goff[g]] for every g: first entry of each graph
__global__ void k_graph_entries(int32_t G, const int32_t *goff, const int32_t *rp, int32_t *eoff) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g <= G; g += gridDim.x * blockDim.x)
        eoff[g] = rp[goff[g]];
}

std::vector<int32_t> graph_entry_offsets(int32_t G, const int32_t *goff_d, const int32_t *rp,
                                         cudaStream_t st) {
    DevBuf e(4 * ((size_t)G + 1), st);
    k_graph_entries<<<slm::grid_for(G + 1, 256), 256, 0, st>>>(G, goff_d, rp, e.as<int32_t>());
    SLM_LAUNCH_CHECK();
    std::vector<int32_t> h((size_t)G + 1);
    SLM_CUDA(cudaMemcpyAsync(h.data(), e.get(), 4 * h.size(), cudaMemcpyDeviceToHost, st));
    slm::stream_sync(st);
    return h;
}

template <class T> void to_device(DevBuf &d, const std::vector<T> &h, cudaStream_t st) {
    d.ensure(sizeof(T) * (h.size() ? h.size() : 1), st);
    if (!h.empty()) SLM_CUDA(cudaMemcpyAsync(d.get(), h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, st));
}

void run_batch(slm_batch *B, const slm_options &opt, cudaStream_t st) {
    using namespace slm;
    if (opt.max_sweeps < 0 || opt.max_sweeps > 65535 || opt.max_levels < 0 ||
        opt.max_levels > 65535 || opt.accept_p32 > (1ull << 32))
        fail(SLM_ERR_INVALID_ARGUMENT, "options out of range");
    const int32_t G = B->G;
    B->has_run = false;
    B->glev.assign(G, {});
    B->gtop.assign(G, slm_level_stats{});
    B->lev_ids.clear();
    B->lev_goff.clear();
    B->lev_koff.clear();
    B->q.assign(G, 0.0);
    B->batch_levels = 0;
    B->batch_sweeps = 0;
    const size_t N0 = (size_t)(B->N0 > 0 ? B->N0 : 1);
    B->final_comp.alloc(4 * N0, st);
    if (B->N0 > 0) {
        k_iota_b<<<grid_for(B->N0, 256), 256, 0, st>>>(B->N0, B->final_comp.as<int32_t>());
        SLM_LAUNCH_CHECK();
    }
    B->final_koff = B->goff0;
    if (G == 0 || B->N0 == 0) {
        B->has_run = true;
        return;
    }
    // per-graph seeds and m_w on the device
    std::vector<unsigned long long> seeds(G, opt.seed);
    if (!B->seeds.empty()) seeds = B->seeds;
    DevBuf seeds_d, goff_d, active_d, done_d, cand_d, pg_d, spl_d, Kg_d, gid_d;
    to_device(seeds_d, seeds, st);
    std::vector<int32_t> goff = B->goff0;
    std::vector<int32_t> done(G, 0);
    to_device(goff_d, goff, st);
    gid_d.alloc(4 * N0, st);
    SLM_CUDA(cudaMemcpyAsync(gid_d.get(), B->gid0.get(), 4 * (size_t)B->N0, cudaMemcpyDeviceToDevice, st));
    int32_t n = B->N0;
    const int32_t *rp = B->rp.as<int32_t>(), *col = B->col.as<int32_t>(), *w = B->w.as<int32_t>();
    const int32_t *s = B->s.as<int32_t>();
    DevBuf lrp, lcol, lw, ls;
    HostCounters hc;
    Work W;
    std::vector<int32_t> active(G), cand(G), pg(2 * (size_t)G), spl(G), Kg(G);
    for (int t = 0;; t++) {
        W.init(n, rp, st);
        const MParam mp(gid_d.as<int32_t>(), B->mg_d.as<long long>());
        RngParam rng(opt.seed);
        rng.gid = gid_d.as<int32_t>();
        rng.seeds = seeds_d.as<unsigned long long>();
        rng.goff = goff_d.as<int32_t>();
        std::vector<int32_t> eoff = graph_entry_offsets(G, goff_d.as<int32_t>(), rp, st);
        std::vector<slm_level_stats> sl(G);
        for (int g = 0; g < G; g++) {
            sl[g].n = goff[g + 1] - goff[g];
            sl[g].nnz = eoff[g + 1] - eoff[g];
        }
        spl_d.ensure(4 * (size_t)G, st);
        SLM_CUDA(cudaMemsetAsync(spl_d.get(), 0, 4 * (size_t)G, st));
        // ASSIGN, COMPONENTS, POSITIVE over the whole forest
        assign_nodes<NMSym>(n, rp, col, w, s, mp, W.bk, W.a.as<int32_t>(), st);
        forest_analyse(n, W.a.as<int32_t>(), W.f, st);
        long long rounds = 0, visits = 0;
        if (!(opt.flags & SLM_FLAG_NO_POSITIVE))
            positive_correct<NMSym>(n, rp, col, w, s, mp, W.a.as<int32_t>(), W.f, W.sigma.as<int32_t>(), W.bk,
                             W.ps, st, &rounds, &visits, spl_d.as<int32_t>());
        int nactive = 0;
        for (int g = 0; g < G; g++) {
            active[g] = done[g] ? 0 : 1;
            nactive += active[g];
            sl[g].status = 2;
            sl[g].sweeps = 0;
        }
        long long bucket_nodes = n;  // nodes the degree buckets cover
        for (int sweep = 0; sweep < opt.max_sweeps && nactive > 0; sweep++) {
            B->batch_sweeps++;
            to_device(active_d, active, st);
            // once the graphs still running hold under half of the nodes the
            // buckets cover, the buckets are rebuilt over their nodes only, so
            // the scans skip the graphs that have stopped
            long long act_nodes = 0;
            for (int g = 0; g < G; g++)
                if (active[g]) act_nodes += goff[g + 1] - goff[g];
            if (2 * act_nodes < bucket_nodes) {
                const int32_t cnt = compact_members(n, nullptr, gid_d.as<int32_t>(), active_d.as<int32_t>(),
                                                    W.alist.as<int32_t>(), W.amark, W.atot, st);
                W.bk.build_list(cnt, W.alist.as<int32_t>(), rp, st);
                bucket_nodes = cnt;
            }
            unsigned long long *ctr = W.ctr();
            SLM_CUDA(cudaMemsetAsync(ctr, 0, 64, st));
            community_sigma(n, W.f.root, s, W.sigma.as<int32_t>(), st);
            scan_nodes<NMSym>(n, rp, col, w, s, mp, W.f.root, W.sigma.as<int32_t>(), W.bk,
                       W.best.as<int32_t>(), W.gain.as<long long>(), W.kown.as<int32_t>(), ctr, st);
            cand_d.ensure(4 * (size_t)G, st);
            SLM_CUDA(cudaMemsetAsync(cand_d.get(), 0, 4 * (size_t)G, st));
            candidates_per_graph(n, gid_d.as<int32_t>(), active_d.as<int32_t>(), W.gain.as<long long>(),
                                 cand_d.as<int32_t>(), st);
            SLM_CUDA(cudaMemcpyAsync(cand.data(), cand_d.get(), 4 * (size_t)G, cudaMemcpyDeviceToHost, st));
            slm::stream_sync(st);
            int still = 0;
            for (int g = 0; g < G; g++) {
                if (!active[g]) continue;
                sl[g].candidates += cand[g];
                sl[g].edges_scanned += sl[g].nnz;
                if (cand[g] == 0) {  // converged
                    sl[g].status = 0;
                    sl[g].sweeps = sweep + 1;
                    active[g] = 0;
                } else still++;
            }
            nactive = still;
            if (nactive == 0) break;
            to_device(active_d, active, st);
            branch_gains<NMSym>(n, rp, col, w, s, mp, W.a.as<int32_t>(), W.f, W.sigma.as<int32_t>(),
                         W.best.as<int32_t>(), W.gain.as<long long>(), W.kown.as<int32_t>(), W.bs,
                         W.bg.as<long long>(), st);
            pg_d.ensure(8 * (size_t)G, st);
            SLM_CUDA(cudaMemsetAsync(pg_d.get(), 0, 8 * (size_t)G, st));
            int32_t *acc_cnt = reinterpret_cast<int32_t *>(ctr + 2);
            accept_moves(n, W.bg.as<long long>(), rng, opt.accept_p32, t, sweep, W.acclist.as<int32_t>(),
                         acc_cnt, ctr + 1, st, active_d.as<int32_t>(), pg_d.as<int32_t>());
            SLM_CUDA(cudaMemcpyAsync(pg.data(), pg_d.get(), 8 * (size_t)G, cudaMemcpyDeviceToHost, st));
            SLM_CUDA(cudaMemcpyAsync(hc.h, ctr, 24, cudaMemcpyDeviceToHost, st));
            slm::stream_sync(st);
            const int32_t nacc = (int32_t)(hc.h[2] & 0xffffffff);
            still = 0;
            for (int g = 0; g < G; g++) {
                if (!active[g]) continue;
                if (pg[2 * g] == 0) {  // stalled: no candidate with a positive branch gain
                    sl[g].status = 1;
                    sl[g].sweeps = sweep + 1;
                    active[g] = 0;
                } else {
                    sl[g].moves += pg[2 * g + 1];
                    still++;
                }
            }
            nactive = still;
            if (nacc > 0) {
                target_nodes<NMSym>(W.acclist.as<int32_t>(), acc_cnt, nacc, rp, col, w, s, mp, W.f.root,
                             W.best.as<int32_t>(), W.tgt.as<int32_t>(), st);
                apply_moves(W.acclist.as<int32_t>(), acc_cnt, nacc, W.tgt.as<int32_t>(),
                            W.a.as<int32_t>(), st);
                // as in slm_run: the components change only in the communities
                // the write touched, and only those can hold a negative local gain
                SLM_CUDA(cudaMemcpyAsync(W.prev_root.get(), W.f.root, 4 * (size_t)n,
                                         cudaMemcpyDeviceToDevice, st));
                const int32_t na = 16LL * nacc > n ? n
                                   : moved_members(n, W.acclist.as<int32_t>(), acc_cnt, nacc, W.f.root,
                                                   W.best.as<int32_t>(), W.alist.as<int32_t>(), W.amark,
                                                   W.ascratch, W.atot, st);
                if (2LL * na > n) forest_analyse(n, W.a.as<int32_t>(), W.f, st);
                else forest_analyse_subset(na, W.alist.as<int32_t>(), W.a.as<int32_t>(), W.f, st);
                if (!(opt.flags & SLM_FLAG_NO_POSITIVE))
                    positive_correct<NMSym>(n, rp, col, w, s, mp, W.a.as<int32_t>(), W.f, W.sigma.as<int32_t>(),
                                     W.bk, W.ps, st, &rounds, &visits, spl_d.as<int32_t>(),
                                     16LL * nacc <= n ? W.prev_root.as<int32_t>() : nullptr);
            }
            if (sweep + 1 == opt.max_sweeps)
                for (int g = 0; g < G; g++)
                    if (active[g]) sl[g].sweeps = sweep + 1;  // status stays 2: sweep limit
        }
        if (opt.flags & SLM_FLAG_STRICT)
            for (int g = 0; g < G; g++)
                if (!done[g] && sl[g].status == 2) fail(SLM_ERR_NOT_CONVERGED, "sweep limit reached");
        SLM_CUDA(cudaMemcpyAsync(spl.data(), spl_d.get(), 4 * (size_t)G, cudaMemcpyDeviceToHost, st));
        // compaction; names per graph
        DevBuf id(4 * (size_t)n, st), scratch(4 * (size_t)n, st);
        compact_labels(n, W.f.root, id.as<int32_t>(), scratch.as<int32_t>(), st);
        Kg_d.ensure(4 * (size_t)G, st);
        SLM_CUDA(cudaMemsetAsync(Kg_d.get(), 0, 4 * (size_t)G, st));
        roots_per_graph(n, W.f.root, gid_d.as<int32_t>(), Kg_d.as<int32_t>(), st);
        SLM_CUDA(cudaMemcpyAsync(Kg.data(), Kg_d.get(), 4 * (size_t)G, cudaMemcpyDeviceToHost, st));
        slm::stream_sync(st);
        bool recorded = false;
        long long dropped = 0;
        for (int g = 0; g < G; g++) {
            if (done[g]) {
                dropped += sl[g].nnz;
                continue;
            }
            sl[g].splits = spl[g];
            sl[g].n_communities = Kg[g];
            if (Kg[g] == sl[g].n) {
                done[g] = 1;
                B->gtop[g] = sl[g];
                dropped += sl[g].nnz;
            } else {
                B->glev[g].push_back({sl[g].n, Kg[g], sl[g]});
                recorded = true;
            }
        }
        if (!recorded) break;
        std::vector<int32_t> koff((size_t)G + 1, 0);
        for (int g = 0; g < G; g++) koff[g + 1] = koff[g] + Kg[g];
        const int32_t K = koff[G];
        compose_labels(B->N0, B->final_comp.as<int32_t>(), id.as<int32_t>(), st);
        B->final_koff = koff;
        B->lev_goff.push_back(goff);
        B->lev_koff.push_back(koff);
        B->batch_levels = t + 1;
        // AGGREGATE, leaving out the rows of the finished graphs
        to_device(done_d, done, st);
        DevBuf nrp, ncol, nw;
        aggregate_graph(n, rp, col, w, id.as<int32_t>(), K, nrp, ncol, nw, st, gid_d.as<int32_t>(),
                        done_d.as<int32_t>(), dropped);
        B->lev_ids.push_back(std::move(id));
        DevBuf ns(4 * (size_t)(K > 0 ? K : 1), st);
        strengths(K, nrp.as<int32_t>(), nw.as<int32_t>(), ns.as<int32_t>(), st);
        lrp = std::move(nrp);
        lcol = std::move(ncol);
        lw = std::move(nw);
        ls = std::move(ns);
        rp = lrp.as<int32_t>();
        col = lcol.as<int32_t>();
        w = lw.as<int32_t>();
        s = ls.as<int32_t>();
        n = K;
        goff = koff;
        to_device(goff_d, goff, st);
        gid_d.ensure(4 * (size_t)(n > 0 ? n : 1), st);
        graph_of_nodes(n, goff_d.as<int32_t>(), G, gid_d.as<int32_t>(), st);
        if (t + 1 >= opt.max_levels) {
            // graphs still running stop here with their last level recorded
            break;
        }
    }
    // final modularity of every graph on its input graph
    DevBuf koff_d, nums_d(8 * (size_t)G, st);
    to_device(koff_d, B->final_koff, st);
    modularity_forest(B->N0, B->rp.as<int32_t>(), B->col.as<int32_t>(), B->w.as<int32_t>(),
                      B->final_comp.as<int32_t>(), B->final_koff[G], B->gid0.as<int32_t>(),
                      koff_d.as<int32_t>(), G, B->mg_d.as<long long>(), nums_d.as<long long>(), st);
    std::vector<long long> nums(G);
    SLM_CUDA(cudaMemcpyAsync(nums.data(), nums_d.get(), 8 * (size_t)G, cudaMemcpyDeviceToHost, st));
    slm::stream_sync(st);
    for (int g = 0; g < G; g++) B->q[g] = modularity_from_num(nums[g], B->mg[g]);
    B->has_run = true;
}

}  // namespace

extern "C" {

slm_status slm_batch_create(int32_t num_graphs, const int32_t *graph_off, const int32_t *row_ptr,
                            const int32_t *col_idx, const int32_t *weights, const uint64_t *seeds,
                            int where, void *stream, slm_batch **out) {
    if (!out) return SLM_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    auto B = std::make_unique<slm_batch>();
    slm_status st = guarded_b(nullptr, [&] {
        using namespace slm;
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        if (num_graphs < 0 || !graph_off || !row_ptr || (where != SLM_HOST && where != SLM_DEVICE))
            fail(SLM_ERR_INVALID_ARGUMENT, "bad num_graphs, graph_off, row_ptr or where");
        const int32_t G = num_graphs;
        B->G = G;
        B->goff0.assign(graph_off, graph_off + G + 1);
        if (B->goff0[0] != 0) fail(SLM_ERR_INVALID_ARGUMENT, "graph_off[0] must be 0");
        for (int g = 0; g < G; g++)
            if (B->goff0[g + 1] < B->goff0[g]) fail(SLM_ERR_INVALID_ARGUMENT, "graph_off must be non-decreasing");
        const int32_t N = B->goff0[G];
        B->N0 = N;
        if (seeds) B->seeds.assign(seeds, seeds + G);
        std::vector<int32_t> rp_h((size_t)N + 1);
        cudaMemcpyKind kind = where == SLM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
        if (where == SLM_HOST) std::memcpy(rp_h.data(), row_ptr, 4 * rp_h.size());
        else {
            SLM_CUDA(cudaMemcpyAsync(rp_h.data(), row_ptr, 4 * rp_h.size(), cudaMemcpyDeviceToHost, s));
            slm::stream_sync(s);
        }
        if (rp_h[0] != 0) fail(SLM_ERR_INVALID_ARGUMENT, "row_ptr[0] must be 0");
        for (int32_t i = 0; i < N; i++)
            if (rp_h[i + 1] < rp_h[i]) fail(SLM_ERR_INVALID_ARGUMENT, "row_ptr must be non-decreasing");
        const long long nnz = rp_h[N];
        if (nnz > 0 && !col_idx) fail(SLM_ERR_INVALID_ARGUMENT, "col_idx is NULL");
        B->nnz0 = (int32_t)nnz;
        B->rp.alloc(4 * ((size_t)N + 1), s);
        B->col.alloc(4 * (size_t)(nnz > 0 ? nnz : 1), s);
        B->w.alloc(4 * (size_t)(nnz > 0 ? nnz : 1), s);
        B->s.alloc(4 * (size_t)(N > 0 ? N : 1), s);
        B->gid0.alloc(4 * (size_t)(N > 0 ? N : 1), s);
        B->mg_d.alloc(8 * (size_t)(G > 0 ? G : 1), s);
        SLM_CUDA(cudaMemcpyAsync(B->rp.get(), rp_h.data(), 4 * rp_h.size(), cudaMemcpyHostToDevice, s));
        if (nnz > 0) {
            SLM_CUDA(cudaMemcpyAsync(B->col.get(), col_idx, 4 * (size_t)nnz, kind, s));
            if (weights) SLM_CUDA(cudaMemcpyAsync(B->w.get(), weights, 4 * (size_t)nnz, kind, s));
            else {
                k_ones_b<<<grid_for(nnz, 256), 256, 0, s>>>(nnz, B->w.as<int32_t>());
                SLM_LAUNCH_CHECK();
            }
        }
        int bad = validate_csr(N, nnz, B->rp.as<int32_t>(), B->col.as<int32_t>(), B->w.as<int32_t>(), s);
        if (bad & (1 | 8)) fail(SLM_ERR_INVALID_ARGUMENT, "column index out of range, unsorted or duplicated");
        if (bad & 2) fail(SLM_ERR_INVALID_ARGUMENT, "non-positive weight");
        if (bad & 4) fail(SLM_ERR_NOT_SYMMETRIC, "W is not symmetric");
        long long mall = strengths(N, B->rp.as<int32_t>(), B->w.as<int32_t>(), B->s.as<int32_t>(), s);
        (void)mall;
        to_device(B->goff0_d, B->goff0, s);
        graph_of_nodes(N, B->goff0_d.as<int32_t>(), G, B->gid0.as<int32_t>(), s);
        long long cross = forest_check_and_weights(N, B->rp.as<int32_t>(), B->col.as<int32_t>(),
                                                   B->s.as<int32_t>(), B->gid0.as<int32_t>(), G,
                                                   B->mg_d.as<long long>(), s);
        if (cross) fail(SLM_ERR_INVALID_ARGUMENT, "an entry joins two different graphs");
        B->mg.resize(G);
        if (G > 0)
            SLM_CUDA(cudaMemcpyAsync(B->mg.data(), B->mg_d.get(), 8 * (size_t)G, cudaMemcpyDeviceToHost, s));
        slm::stream_sync(s);
        for (int g = 0; g < G; g++)
            if (B->mg[g] >= (1LL << 31)) fail(SLM_ERR_OVERFLOW, "a graph's m_w is not below 2^31");
    });
    if (st == SLM_OK) *out = B.release();
    return st;
}

slm_status slm_batch_run(slm_batch *b, const slm_options *opt, void *stream) {
    if (!b) return SLM_ERR_INVALID_ARGUMENT;
    slm_options o;
    slm_default_options(&o);
    if (opt) o = *opt;
    return guarded_b(b, [&] { run_batch(b, o, reinterpret_cast<cudaStream_t>(stream)); });
}

slm_status slm_batch_num_graphs(const slm_batch *b, int32_t *num_graphs) {
    if (!b || !num_graphs) return SLM_ERR_INVALID_ARGUMENT;
    *num_graphs = b->G;
    return SLM_OK;
}

slm_status slm_batch_num_levels(const slm_batch *b, int32_t graph, int32_t *levels) {
    if (!b || !levels || graph < 0 || graph >= b->G) return SLM_ERR_INVALID_ARGUMENT;
    if (!b->has_run) return SLM_ERR_NOT_RUN;
    *levels = (int32_t)b->glev[graph].size();
    return SLM_OK;
}

slm_status slm_batch_get_partition(const slm_batch *b, int32_t graph, int32_t level,
                                   int32_t *labels, int32_t *n_communities) {
    if (!b || graph < 0 || graph >= b->G) return SLM_ERR_INVALID_ARGUMENT;
    if (!b->has_run) return SLM_ERR_NOT_RUN;
    const int32_t L = (int32_t)b->glev[graph].size();
    if (level < -1 || level >= L) return SLM_ERR_INVALID_ARGUMENT;
    slm_batch *bm = const_cast<slm_batch *>(b);
    return guarded_b(bm, [&] {
        int32_t lo, hi, base, K;
        const slm::DevBuf *src;
        if (level == -1) {
            lo = b->goff0[graph];
            hi = b->goff0[graph + 1];
            base = b->final_koff[graph];
            K = b->final_koff[graph + 1] - b->final_koff[graph];
            src = &b->final_comp;
        } else {
            lo = b->lev_goff[level][graph];
            hi = b->lev_goff[level][graph + 1];
            base = b->lev_koff[level][graph];
            K = b->glev[graph][level].K;
            src = &b->lev_ids[level];
        }
        if (hi > lo) {
            if (!labels) slm::fail(SLM_ERR_INVALID_ARGUMENT, "labels is NULL");
            SLM_CUDA(cudaMemcpy(labels, src->as<int32_t>() + lo, 4 * (size_t)(hi - lo), cudaMemcpyDeviceToHost));
            for (int32_t k = 0; k < hi - lo; k++) labels[k] -= base;
        }
        if (n_communities) *n_communities = K;
    });
}

slm_status slm_batch_modularity(const slm_batch *b, int32_t graph, double *q) {
    if (!b || !q || graph < 0 || graph >= b->G) return SLM_ERR_INVALID_ARGUMENT;
    if (!b->has_run) return SLM_ERR_NOT_RUN;
    *q = b->q[graph];
    return SLM_OK;
}

slm_status slm_batch_get_stats(const slm_batch *b, int32_t graph, int32_t level, slm_level_stats *st) {
    if (!b || !st || graph < 0 || graph >= b->G) return SLM_ERR_INVALID_ARGUMENT;
    if (!b->has_run) return SLM_ERR_NOT_RUN;
    const int32_t L = (int32_t)b->glev[graph].size();
    if (level < -1 || level >= L) return SLM_ERR_INVALID_ARGUMENT;
    *st = level == -1 ? b->gtop[graph] : b->glev[graph][level].st;
    return SLM_OK;
}

slm_status slm_batch_run_info(const slm_batch *b, int32_t *batch_levels, int64_t *batch_sweeps) {
    if (!b || !batch_levels || !batch_sweeps) return SLM_ERR_INVALID_ARGUMENT;
    if (!b->has_run) return SLM_ERR_NOT_RUN;
    *batch_levels = b->batch_levels;
    *batch_sweeps = b->batch_sweeps;
    return SLM_OK;
}

void slm_batch_destroy(slm_batch *b) {
    if (!b) return;
    slm::ReleaseOnDefaultStream on_default;
    delete b;
}

const char *slm_batch_last_error(const slm_batch *b) {
    return b ? b->err.c_str() : g_batch_create_error.c_str();
}

}  // extern "C"
