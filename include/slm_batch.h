/*
 * slm_batch.h -- many independent graphs in one run.
 *
 * A forest is one block-diagonal symmetric CSR: graph g owns the global node
 * range [graph_off[g], graph_off[g+1]) and every stored entry joins two nodes
 * of the same graph.  slm_batch_run applies Algorithm 1 of the paper
 * (Section 3) to every graph at once: each level's kernels cover all the
 * graphs still running, with the modularity of each graph (Section 2.4, its
 * own m_w), its own seed and sweep control, and its own stopping rules.  A
 * graph's partitions, statistics and modularity are bit for bit those of
 * slm_run on that graph alone with that seed: nothing in a graph's
 * arithmetic depends on the other graphs.
 *
 * Conventions as in slm.h (status codes, `where`, copied inputs, the stream).
 */
#ifndef SLM_BATCH_H
#define SLM_BATCH_H

#include "slm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct slm_batch slm_batch; /* opaque, owned by the library */

/* Copy and validate a forest.  graph_off (HOST, num_graphs+1 entries,
 * graph_off[0] = 0, non-decreasing) gives the node ranges; row_ptr
 * (graph_off[G]+1 entries), col_idx and weights (NULL: unit) are in `where`
 * memory with global node ids; seeds (HOST, num_graphs entries, NULL: the
 * run's opt.seed for every graph) key each graph's acceptance draws.
 * Limits: node ids and entry offsets are int32 over the whole forest, so the
 * forest holds fewer than 2^31 nodes and fewer than 2^31 stored entries in
 * all (row_ptr[graph_off[G]] < 2^31); a larger set of graphs is run as
 * several forests.  Every node id in col_idx is global (graph g's nodes are
 * graph_off[g] .. graph_off[g+1]-1), while results are reported with each
 * graph's own local ids.
 * Errors: INVALID_ARGUMENT (bad offsets, CSR, or an entry joining two
 * graphs), NOT_SYMMETRIC, OVERFLOW (some graph's m_w >= 2^31),
 * OUT_OF_MEMORY, CUDA. */
slm_status slm_batch_create(int32_t num_graphs, const int32_t *graph_off, const int32_t *row_ptr,
                            const int32_t *col_idx, const int32_t *weights, const uint64_t *seeds,
                            int where, void *stream, slm_batch **out);

/* Run the method on every graph (opt as for slm_run; opt.seed is used for the
 * graphs without a seed).  Returns when the run has finished on `stream`. */
slm_status slm_batch_run(slm_batch *b, const slm_options *opt, void *stream);

slm_status slm_batch_num_graphs(const slm_batch *b, int32_t *num_graphs);
/* Recorded levels of one graph. */
slm_status slm_batch_num_levels(const slm_batch *b, int32_t graph, int32_t *levels);
/* Partition of one graph at one of its levels (its level-t node count of
 * labels, ids local to the graph, 0..K-1), or level = -1 the final partition
 * of the graph's input nodes.  labels: HOST memory.  Synchronous. */
slm_status slm_batch_get_partition(const slm_batch *b, int32_t graph, int32_t level,
                                   int32_t *labels, int32_t *n_communities);
/* Final modularity of one graph (computed on the device at the end of the run). */
slm_status slm_batch_modularity(const slm_batch *b, int32_t graph, double *q);
/* Statistics of one graph's level (level = -1: its last, unrecorded level). */
slm_status slm_batch_get_stats(const slm_batch *b, int32_t graph, int32_t level,
                               slm_level_stats *st);
/* Kernel-level summary of the last run: levels of the whole batch and sweeps
 * launched (each sweep covers every graph still running). */
slm_status slm_batch_run_info(const slm_batch *b, int32_t *batch_levels, int64_t *batch_sweeps);
void slm_batch_destroy(slm_batch *b);
const char *slm_batch_last_error(const slm_batch *b);

#ifdef __cplusplus
}
#endif
#endif /* SLM_BATCH_H */
