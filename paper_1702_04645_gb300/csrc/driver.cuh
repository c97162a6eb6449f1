// driver.cuh -- the per-level device workspace shared by the host drivers
// (one graph: slm_api.cu; a forest of graphs: slm_batch.cu).
#pragma once

#include "slm_internal.cuh"

namespace slm {

// Per-level device workspace: every array sized for the level's n, grown on demand.
struct Work {
    int32_t n = 0;
    DevBuf a, sigma, best, kown, tgt, acclist, gain, bg, counters;
    DevBuf root, oncycle, entry, depth, cdist, jmpA, jmpB;
    DevBuf prev_root;  // community names after the last POSITIVE
    DevBuf alist, amark, ascratch, atot;  // nodes of the communities a write touched
    DevBuf bs_i32, bs_i64;
    slm::Forest f;
    slm::BranchScratch bs{};
    slm::PositiveScratch ps;
    slm::Buckets bk;

    void init(int32_t n_, const int32_t *rp, cudaStream_t st) {
        n = n_;
        size_t N = (size_t)(n > 0 ? n : 1);
        a.ensure(4 * N, st);
        sigma.ensure(8 * N, st);  // int32 totals, or packed (out, in) pairs of a directed graph
        best.ensure(4 * N, st);
        kown.ensure(4 * N, st);
        tgt.ensure(4 * N, st);
        acclist.ensure(4 * N, st);
        gain.ensure(8 * N, st);
        bg.ensure(8 * N, st);
        counters.ensure(64, st);
        root.ensure(4 * N, st);
        prev_root.ensure(4 * N, st);
        alist.ensure(4 * N, st);
        oncycle.ensure(N, st);
        entry.ensure(4 * N, st);
        depth.ensure(4 * N, st);
        cdist.ensure(4 * N, st);
        jmpA.ensure(8 * N, st);
        jmpB.ensure(8 * N, st);
        bs_i32.ensure(4 * N * 5, st);
        bs_i64.ensure(8 * N * 5, st);
        f.root = root.as<int32_t>();
        f.oncycle = oncycle.as<uint8_t>();
        f.entry = entry.as<int32_t>();
        f.depth = depth.as<int32_t>();
        f.cdist = cdist.as<int32_t>();
        f.jmpA = jmpA.as<int2>();
        f.jmpB = jmpB.as<int2>();
        int32_t *p32 = bs_i32.as<int32_t>();
        long long *p64 = bs_i64.as<long long>();
        bs.haschild = p32;
        bs.active = p32 + N;
        bs.covered = p32 + 2 * N;
        bs.treeact = p32 + 3 * N;
        bs.commcyc = p32 + 4 * N;
        bs.subS = p64;
        bs.subWA = p64 + N;
        bs.subWin = p64 + 2 * N;
        bs.credit = p64 + 3 * N;
        bs.WB = p64 + 4 * N;
        bk.build(n, rp, st);
    }
    unsigned long long *ctr() { return counters.as<unsigned long long>(); }
};

}  // namespace slm
