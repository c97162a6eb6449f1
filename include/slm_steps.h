/*
 * slm_steps.h -- one C entry point per step of the Synchronised Louvain
 * Method, on caller-owned DEVICE buffers.  They run the same kernels that
 * slm_run chains together and exist so that every step can be checked alone
 * against a reference on identical inputs.
 *
 * Shared conventions:
 *   - every pointer argument is device memory of the current device unless
 *     its name ends in `_host`;
 *   - graphs are symmetric CSR (row_ptr int32[n+1], col int32[nnz] sorted
 *     unique per row, w int32[nnz] > 0); s is int32[n] (s_i = sum_j W_ij) and
 *     m_w = sum_i s_i < 2^31;
 *   - "names" of communities are node ids: a community is named by the
 *     smallest node on its assignment cycle (root[v] in [0, n));
 *   - scratch memory is allocated with cudaMallocAsync on `stream` and freed
 *     before return; every function synchronises `stream` before returning;
 *   - errors: SLM_ERR_INVALID_ARGUMENT for negative sizes or NULL pointers
 *     with a non-zero size, SLM_ERR_OUT_OF_MEMORY, SLM_ERR_CUDA.
 */
#ifndef SLM_STEPS_H
#define SLM_STEPS_H

#include "slm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Strengths s_i = sum_j W_ij and m_w = sum_i s_i (Section 2.4, m_w). */
slm_status slm_step_strengths(int32_t n, const int32_t *row_ptr, const int32_t *col,
                              const int32_t *w, int32_t *s, int64_t *m_w_host, void *stream);

/* ASSIGN (Section 3.1, Algorithm ASSIGN): a[i] = argmax over neighbours j != i
 * of m_w W_ij - s_i s_j, smallest j on ties, a[i] = i when no value is > 0. */
slm_status slm_step_assign(int32_t n, const int32_t *row_ptr, const int32_t *col,
                           const int32_t *w, const int32_t *s, int64_t m_w, int32_t *a,
                           void *stream);

/* COMPONENTS (Section 3.2): root[v] = smallest node on the cycle that v's
 * forward path in the assignment graph a reaches.  a[v] in [0, n). */
slm_status slm_step_components(int32_t n, const int32_t *a, int32_t *root, void *stream);

/* The per-node scan of MAXIMAL (Section 3.4, best community c_i^*):
 * Sigma_C = sum of s over community C; for every node i,
 * score(C) = m_w k_{i,C} - s_i (Sigma_C - [C = root_i] s_i) with k_{i,C} the
 * weight from i to C (self-loop excluded); best[i] = the neighbouring
 * community C != root_i of largest score (smallest name on ties) when
 * gain[i] = score(best) - score(root_i) > 0, else best[i] = root[i] and
 * gain[i] = 0; g[i] = score(root_i) is the local gain of Algorithm POSITIVE. */
slm_status slm_step_scan(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *w,
                         const int32_t *s, int64_t m_w, const int32_t *root, int32_t *best,
                         int64_t *gain, int64_t *g, void *stream);

/* Branch gain of Algorithm MAXIMAL for every node with gain[i] > 0 (bg[i] = 0
 * elsewhere): moving the tail S of i (every node whose forward path reaches i)
 * from A = root_i to B = best_i changes the modularity numerator by twice
 *   m_w (W(S,B) - W(S, A\S)) - Sigma_S (Sigma_B - Sigma_A + Sigma_S).
 * root must be the components of a; best and gain as produced by the scan. */
slm_status slm_step_branch_gain(int32_t n, const int32_t *row_ptr, const int32_t *col,
                                const int32_t *w, const int32_t *s, int64_t m_w,
                                const int32_t *a, const int32_t *root, const int32_t *best,
                                const int64_t *gain, int64_t *bg, void *stream);

/* One synchronous MAXIMAL correction (Algorithm MAXIMAL, Section 4.2): scan,
 * branch gains, the random acceptance draw of level `level`, sweep `sweep`,
 * the target node a'(i) = argmax over neighbours j of i in best_i of
 * m_w W_ij - s_i s_j (smallest j on ties), and one simultaneous write of a'.
 * a is updated in place; root (the components of a on entry) is left as is.
 * counts_host[0..2] = candidates (gain > 0), candidates with a positive
 * branch gain, accepted moves. */
slm_status slm_step_maximal(int32_t n, const int32_t *row_ptr, const int32_t *col,
                            const int32_t *w, const int32_t *s, int64_t m_w, int32_t *a,
                            const int32_t *root, uint64_t seed, uint64_t accept_p32,
                            int32_t level, int32_t sweep, int64_t *counts_host, void *stream);

/* POSITIVE (Section 3.3, Algorithm POSITIVE): bisect every community that
 * holds a node with a negative local gain, optimally over the branch cuts
 * and the two-node cycle cuts of its assignment graph (largest value of
 * Sigma_S Sigma_R - m_w W(S,R); ties: branch before cycle, then smaller u,
 * then smaller v), and repeat on the parts until no node has a negative local
 * gain.  a is updated in place; root receives the final components. */
slm_status slm_step_positive(int32_t n, const int32_t *row_ptr, const int32_t *col,
                             const int32_t *w, const int32_t *s, int64_t m_w, int32_t *a,
                             int32_t *root, int64_t *splits_host, void *stream);

/* Compaction: id[v] = rank of root[v] among the names in use (root[x] == x),
 * *K_host = their number. */
slm_status slm_step_compact(int32_t n, const int32_t *root, int32_t *id, int32_t *K_host,
                            void *stream);

/* AGGREGATE (Section 3.5): W'_AB = sum of W_uv over id[u] = A, id[v] = B,
 * diagonal included, as a CSR with sorted unique columns.  row_ptr_out holds
 * K+1 entries, col_out and w_out at least nnz; *nnz_out_host receives the
 * entries written.  Keys (id[u], id[v]) are sorted by a radix sort and
 * reduced by segment. */
slm_status slm_step_aggregate(int32_t n, const int32_t *row_ptr, const int32_t *col,
                              const int32_t *w, const int32_t *id, int32_t K,
                              int32_t *row_ptr_out, int32_t *col_out, int32_t *w_out,
                              int32_t *nnz_out_host, void *stream);

/* Modularity Q_w (Section 2.4) of labels (values in [0, n)): the exact
 * numerator sum_C (m_w W_in(C) - Sigma_C^2) into *num_host and its FP64
 * quotient by m_w^2 into *q_host (0 when m_w = 0). */
slm_status slm_step_modularity(int32_t n, const int32_t *row_ptr, const int32_t *col,
                               const int32_t *w, const int32_t *labels, double *q_host,
                               int64_t *num_host, void *stream);

/* Modularity of labels without any device allocation, for callers that
 * cannot let a library call cudaMalloc (for instance a framework that has
 * handed all device memory to its own caching allocator or arena and forbids
 * further allocations in the middle of its work).  The paper has no
 * counterpart: this is the computation of slm_step_modularity with its
 * scratch moved into one fixed, file-scope device array of 2^21 + 4 words
 * (16 MiB), which every GPU that loads this library holds until the process
 * exits.
 *   - n must not exceed 1048576 (else SLM_ERR_INVALID_ARGUMENT and a message
 *     for slm_last_error(NULL)); labels and columns must lie in [0, n) (else
 *     SLM_ERR_INVALID_ARGUMENT, detected on the device, nothing written
 *     out of bounds);
 *   - *num_out (int64) and *q_out (double) are DEVICE pointers receiving the
 *     exact numerator sum_C (m_w W_in(C) - Sigma_C^2) and its FP64 quotient by
 *     m_w^2 (0 when m_w = 0), the same values slm_step_modularity returns;
 *     when a label or column is found outside [0, n) the call still writes
 *     both outputs (values of the in-range part only) before it returns
 *     SLM_ERR_INVALID_ARGUMENT, so a caller must ignore them then;
 *   - the first call on a device looks up the array's device address (a
 *     cudaGetSymbolAddress with that device current), so make that first call
 *     before any stream capture;
 *   - every call shares the one array and clears what it uses; calls that
 *     overlap on the GPU (two streams, or two threads) race and must not be
 *     issued concurrently;
 *   - the call synchronises `stream` before returning. */
slm_status slm_step_modularity_noalloc(int32_t n, const int32_t *row_ptr, const int32_t *col,
                                       const int32_t *w, const int32_t *labels, int64_t *num_out,
                                       double *q_out, void *stream);

/* Diagnostic record of the last slm_run: one row of six int64 per scan
 * (level, sweep, candidates, candidates with a positive branch gain,
 * accepted moves, POSITIVE splits after the write).  Copies at most `cap`
 * rows into `rows` (host memory) and sets *len to the number of rows. */
slm_status slm_get_trace(const slm_graph *g, int64_t *rows, int64_t cap, int64_t *len);

/* Device time of the phases of the last slm_run made with SLM_FLAG_TIMING,
 * measured with CUDA events on the run's stream: ms8[k] milliseconds over
 * count8[k] intervals for k = 0 assign, 1 components, 2 POSITIVE, 3 scan
 * (accumulate + argmax), 4 branch gains + draw + target + write, 5 level
 * set-up, compaction and aggregation, 6 community totals.  Slot 7 is not a
 * time: count8[7] is the number of POSITIVE rounds and ms8[7] the member
 * visits summed over those rounds. */
slm_status slm_get_timing(const slm_graph *g, double *ms8, int64_t *count8);

/* Device time of the MAXIMAL scans (accumulate + argmax) of one level of the
 * last slm_run made with SLM_FLAG_TIMING (level = -1: the last, unrecorded
 * level): *ms milliseconds over *count scans, CUDA events on the run's
 * stream.  Without SLM_FLAG_TIMING both are 0. */
slm_status slm_get_scan_timing(const slm_graph *g, int32_t level, double *ms, int64_t *count);

/* Device time of the level-0 scans of the last slm_run made with
 * SLM_FLAG_TIMING, split by degree bucket (each bucket's kernels are timed
 * with CUDA events on the stream that runs them; the buckets run side by
 * side on four streams, so the times overlap): ms[k] for buckets
 * 0 isolated, 1 degrees 1-4, 2 5-8, 3 9-16, 4 17-32, 5 33-256 (warp table),
 * 6 257-1024, 7 1025-2048, 8 2049-4096 (block tables), 9 above 4096 (hubs).
 * Copies at most `cap` values and sets *len to the number of buckets. */
slm_status slm_get_scan_bucket_timing(const slm_graph *g, double *ms, int32_t cap, int32_t *len);

/* Profile of the POSITIVE rounds of the last slm_run made with
 * SLM_FLAG_TIMING: nanoseconds of device time per phase of a round, summed
 * over every round of the run, read from the GPU's global timer at the grid
 * barriers that end the phases.  Phases: 0 round set-up, 1 offsets of the
 * member lists (prefix sums), 2 ancestor walks and per-edge credits, 3
 * subtree credits, 4 choice of the best cut (Algorithm POSITIVE, optimal
 * bisection), 5 application of the cuts, 6 new components of the members,
 * 7 local gains g(i), 8 member list of the next round; then two counts
 * rather than times: 9 rounds run on the full grid (the others ran on the
 * small grid that finishes a call), 10 member visits of those rounds.
 * Copies at most `cap` values into `ns` (host memory) and sets *len to the
 * number of values. */
slm_status slm_get_positive_profile(const slm_graph *g, int64_t *ns, int32_t cap, int32_t *len);

/* Self-check of the failure path of the cooperative kernels (POSITIVE runs
 * all its rounds in one launch whose blocks meet at grid barriers; each
 * barrier wait has a time limit, 4 s in POSITIVE, after which the launch is
 * abandoned and slm_run returns SLM_ERR_TIMEOUT).  Launches `blocks` blocks
 * that pass three such barriers with a limit of limit_s seconds (0 < limit_s
 * <= 60); block `absent_block` (-1: none) leaves before the first barrier,
 * so that the other blocks' waits run out.  Returns SLM_OK when every block
 * passed every barrier, SLM_ERR_TIMEOUT when a wait ran out (the device and
 * the context stay usable), SLM_ERR_INVALID_ARGUMENT for a block count that
 * cannot be resident at once.  Synchronous. */
slm_status slm_check_grid_barrier(int32_t blocks, int32_t absent_block, double limit_s,
                                  void *stream);

/* Launch shapes of the MAXIMAL scan, process-wide (no counterpart in the
 * paper; results never depend on them, only speed does).  streams: 1 runs
 * the degree buckets one after another on the caller's stream, 4 runs them
 * side by side on the caller's stream and three library streams; the other
 * fields cap each kernel shape's grid at that many blocks per SM
 * (1..64).  Defaults: {4, 3, 6, 8, 8, 8, 16, 0}. */
typedef struct {
    int32_t streams;
    int32_t blocks_large; /* 2049..4096 edges per node, 64 KB shared table */
    int32_t blocks_mid;   /* 1025..2048 edges, 32 KB table */
    int32_t blocks_small; /* 257..1024 edges, 16 KB table */
    int32_t blocks_warp;  /* 33..256 edges, one warp table per node */
    int32_t blocks_hub;   /* above 4096 edges: row chunks and table slices */
    int32_t blocks_group; /* 1..32 edges: lane groups */
    /* Shape per fine degree class: bit k-1 set selects the second shape of
     * class k (k = 1 for rows of 1..4 entries, 2: 5..8, 3: 9..16, 4: 17..32,
     * 5: 33..64, 6: 65..128, 7: 129..256, 8: 257..512, 9: 513..1024,
     * 10: 1025..2048, 11: 2049..4096).  First / second shape per class:
     * 1: a thread per node / 4 lanes; 2: a thread / 8 lanes; 3: 4 lanes x 4
     * entries / 8 x 2; 4: 8 x 4 / 16 x 2; 5: 16 x 4 / 32 x 2; 6: 32 x 4 / a
     * 64-thread block x 2; 7: 32 x 8 / a 64-thread block x 4; 8: 128-thread
     * blocks x 4 / 256 x 2; 9: 256 x 4 / 512 x 2; 10: 256 x 8 / 512 x 4;
     * 11: 512 x 8 / 1024 x 4.  Classes 6 and 7 thereby move the boundary
     * between the lane-group and the block kernels between 64, 128 and 256
     * entries.  Default 0 (every first shape); 0 <= shape_alt < 2^11. */
    int32_t shape_alt;
} slm_scan_tuning;
/* Set (INVALID_ARGUMENT when a field is out of range) or read the tuning. */
slm_status slm_set_scan_tuning(const slm_scan_tuning *t);
slm_status slm_get_scan_tuning(slm_scan_tuning *t);

/* Number of kernels this library has launched in the process so far. */
uint64_t slm_launch_count(void);

/* Failure injection for tests of the error paths (the paper has no
 * counterpart): the k-th device allocation the library makes from now on, on
 * any thread, fails as if the device were out of memory, so the call that
 * made it returns SLM_ERR_OUT_OF_MEMORY; k = 0 turns the hook off, and it
 * turns itself off once it has fired.  Nothing is done to the device: the
 * allocation is refused on the host before cudaMallocFromPoolAsync is
 * called.  A failed slm_create_graph returns no handle and keeps no memory;
 * a failed slm_run leaves the handle usable, with the results of its
 * previous run (if any). */
void slm_debug_fail_allocation(int64_t k);

#ifdef __cplusplus
}
#endif
#endif /* SLM_STEPS_H */
