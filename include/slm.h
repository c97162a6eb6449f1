/*
 * slm.h -- C ABI of the GB300 implementation of the Synchronised Louvain
 * Method (Chiem, Havelange, Van Dooren, "A parallel implementation of the
 * Synchronised Louvain Method", arXiv:1702.04645, Section 3, Algorithm 1).
 *
 * Input: an undirected graph given as a symmetric CSR with int32 row
 * pointers, int32 column indices sorted ascending and unique in every row,
 * and positive int32 weights (NULL means unit weights); a self-loop W_ii is
 * stored once.  Output: one partition per hierarchical level (Section 3.5)
 * and the final partition of the input nodes (Algorithm 1, C = C_t C).
 *
 * Arithmetic: with s_i = sum_j W_ij and m_w = sum_i s_i, every modularity gain
 * is compared as the exact int64 value m_w * k - s * Sigma (Section 2.4, Q_w),
 * so results are reproducible bit for bit.  m_w must be below 2^31.
 *
 * Conventions for every function:
 *   - the return value is an slm_status; no function aborts or exits;
 *   - `stream` is a cudaStream_t (NULL: the legacy default stream);
 *   - `where` says whether a pointer is host (SLM_HOST) or device (SLM_DEVICE)
 *     memory of the current device;
 *   - inputs are copied; the caller keeps ownership of every pointer it passes;
 *   - the library allocates its device memory in stream order on the given
 *     stream, from a memory pool of its own per device, and frees it in
 *     slm_destroy_graph; freed memory stays cached in that pool for the next
 *     allocation until slm_release_cached_memory returns it to the device.
 */
#ifndef SLM_H
#define SLM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SLM_OK = 0,
    SLM_ERR_INVALID_ARGUMENT = 1, /* bad pointer, size, unsorted/duplicate column, w <= 0 */
    SLM_ERR_NOT_SYMMETRIC = 2,    /* W_ij != W_ji for some pair */
    SLM_ERR_OVERFLOW = 3,         /* m_w >= 2^31: int64 gains would not be exact */
    SLM_ERR_OUT_OF_MEMORY = 4,    /* device allocation failed; state unchanged */
    SLM_ERR_CUDA = 5,             /* a CUDA call failed; see slm_last_error */
    SLM_ERR_NOT_RUN = 6,          /* results asked before slm_run */
    SLM_ERR_NOT_CONVERGED = 7,    /* sweep limit reached and SLM_FLAG_STRICT set */
    SLM_ERR_TIMEOUT = 8,          /* a bounded device-side wait gave up */
    SLM_ERR_BUDGET = 9,           /* a request exceeds the server's whole memory budget */
    SLM_ERR_CANCELLED = 10,       /* a server request was cancelled (slm_server_cancel) */
    SLM_ERR_DEADLINE = 11         /* a server request passed its deadline before it finished */
} slm_status;

#define SLM_HOST 0
#define SLM_DEVICE 1

/* Option flags. */
#define SLM_FLAG_NO_POSITIVE 1u /* skip POSITIVE (ablation; Section 3.3) */
#define SLM_FLAG_STRICT 2u      /* sweep limit reached => SLM_ERR_NOT_CONVERGED */
#define SLM_FLAG_TIMING 4u      /* time the phases of slm_run with CUDA events (see slm_get_timing) */

typedef struct slm_graph slm_graph; /* opaque, owned by the library */

typedef struct {
    /* Seed of the counter-based draw that accepts a maximal correction with
       probability P / 2^32 (Algorithm MAXIMAL, "draw p(i)"; the paper leaves p
       to Browet's thesis, so P is a parameter).  Node i of level t in sweep k
       is accepted iff (mix64(seed ^ mix64(t<<48 | k<<32 | i)) >> 32) < P, with
       mix64 the splitmix64 output function. */
    uint64_t seed;
    uint64_t accept_p32;  /* P in [0, 2^32]; default 2^31 (p = 1/2) */
    int32_t max_sweeps;   /* MAXIMAL+POSITIVE rounds per level (Algorithm 1 inner loop); default 1000, <= 65535 */
    int32_t max_levels;   /* aggregation levels (Algorithm 1 outer loop); default 64, <= 65535 */
    uint32_t flags;       /* SLM_FLAG_* */
} slm_options;

typedef struct {
    int32_t n;              /* nodes of this level's graph */
    int32_t n_communities;  /* K: communities found at this level */
    int32_t sweeps;         /* scans performed by the inner loop */
    int32_t status;         /* 0 converged, 1 stalled (no candidate with a positive branch gain), 2 sweep limit */
    int64_t moves;          /* accepted maximal corrections */
    int64_t splits;         /* positive corrections (bisections) */
    int64_t candidates;     /* nodes with a positive single-node gain, summed over scans */
    int64_t edges_scanned;  /* CSR entries read by the scans (sweeps * nnz) */
    int64_t nnz;            /* stored entries of this level's graph */
} slm_level_stats;

/* Fill *opt with the defaults above. */
void slm_default_options(slm_options *opt);

/* Copy a symmetric CSR graph to the device and validate it (Section 2.4
 * defines s_i and m_w, computed here).  row_ptr has n+1 entries, col_idx and
 * weights row_ptr[n] entries, all in `where` memory.  Errors:
 * INVALID_ARGUMENT, NOT_SYMMETRIC, OVERFLOW, OUT_OF_MEMORY, CUDA.  On success
 * *out owns device copies; destroy it with slm_destroy_graph. */
slm_status slm_create_graph(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                            const int32_t *weights, int where, void *stream, slm_graph **out);

/* A directed graph, the setting of the paper's own experiments (Section 5.1,
 * weighted directed LFR graphs).  W is given as a CSR of out-arcs: row i
 * holds the arcs i -> j with positive weights W_ij, columns sorted ascending
 * and unique per row, no symmetry required (a self-loop W_ii is stored once).
 * The method then optimises Q_w of Section 2.4 with out- and in-strengths:
 *   Q_w = (1/m_w) sum_ij [W_ij - s_i^out s_j^in / m_w] delta(c_i, c_j),
 * with s_i^out = sum_j W_ij, s_j^in = sum_i W_ij and m_w = sum_ij W_ij.  A
 * node's neighbours are the nodes joined to it by an arc either way, and every
 * gain is the exact int64 change of the numerator (the weight term counts
 * U = W + W^T, the null-model term s_i^out Sigma_C^in + s_i^in Sigma_C^out).
 * U and the strengths are built on the host during the call (W in `where`
 * memory is copied there first).  Errors: INVALID_ARGUMENT (CSR shape,
 * column out of range, unsorted or duplicated, w <= 0), OVERFLOW (m_w >= 2^30
 * or more than 2^30 arcs: the packed strength totals and the int64 gains
 * need it), OUT_OF_MEMORY, CUDA.  slm_run, slm_get_partition, slm_modularity
 * (the directed Q_w above), slm_get_stats and slm_destroy_graph take the
 * handle as they take an undirected one. */
slm_status slm_create_graph_directed(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                                     const int32_t *weights, int where, void *stream,
                                     slm_graph **out);
/* 1 for a handle made by slm_create_graph_directed, 0 otherwise. */
int32_t slm_graph_is_directed(const slm_graph *g);

/* Run Algorithm 1 on the graph: per level ASSIGN, COMPONENTS, POSITIVE, then
 * MAXIMAL and POSITIVE alternately until no positive move remains, then
 * AGGREGATE; stop when a level finds no community structure.  On success the
 * results replace those of any previous run; when the run fails (for
 * instance OUT_OF_MEMORY) the handle keeps the previous run's results, if
 * any, and stays usable.  Returns after the work on `stream` has finished
 * (the host reads a few counters per sweep). */
slm_status slm_run(slm_graph *g, const slm_options *opt, void *stream);

/* Colour-synchronous Louvain, the comparison method: classical Louvain's
 * node moves (Section 3, Blondel et al.; leave the own community for the
 * neighbouring one of largest strictly positive gain, ties to the smallest
 * community name) in the parallel form that Section 6 leaves for later work.
 * Per level the nodes get a first-fit colouring in a seeded order (node v at
 * level t has the key mix64(seed ^ mix64((t << 32) | v)), mix64 the
 * splitmix64 output function; larger keys first, equal keys by smaller id;
 * each node takes the smallest colour no earlier neighbour holds; self-loops
 * do not count).  A pass visits the colours 0, 1, ... in turn: all nodes of
 * the colour decide on the communities and totals as they stand, then move at
 * once.  Moves taken together can undo one another's gains, so a level ends
 * at a pass that moves no node (status 0), or that raises the exact numerator
 * sum_C (m_w W_in(C) - Sigma_C^2) by at most floor(m_w^2 / 2^20), i.e. Q by
 * at most 2^-20 (status 1), or after `max_passes` (1..65535) passes (status
 * 2); then the communities are compacted in name order and aggregated as
 * slm_run's are, and the run stops at the first level whose
 * first pass moves nothing or that ends with every node alone, or after
 * `max_levels` (0..65535; at least one level is always run) recorded levels.
 * The results replace the handle's, as slm_run's do (kept on failure), and are
 * read with the same calls; per level slm_level_stats gives sweeps = passes,
 * status (0, 1 or 2 as above), moves, splits =
 * candidates = 0 and edges_scanned = passes x nnz; slm_get_trace (slm_steps.h) gives one row
 * (level, pass, 0, 0, moves, 0) per pass.  A symmetric graph only: a handle
 * from slm_create_graph_directed gives INVALID_ARGUMENT, as do options out of
 * range.  Other errors: OUT_OF_MEMORY, CANCELLED / DEADLINE (run control),
 * CUDA.  Returns after the work on `stream` has finished (the host reads a
 * count per colouring round and per pass). */
slm_status slm_run_louvain(slm_graph *g, uint64_t seed, int32_t max_passes, int32_t max_levels,
                           void *stream);

/* Number of recorded (aggregated) levels of the last run. */
slm_status slm_num_levels(const slm_graph *g, int32_t *levels);

/* Partition of level `level` on that level's nodes (community ids 0..K-1,
 * ordered by the smallest node on each community's assignment cycle), or with
 * level = -1 the final partition composed onto the input nodes.  `labels`
 * must hold n_level (resp. n) int32 in `where` memory; *n_communities gets K.
 * Synchronous. */
slm_status slm_get_partition(const slm_graph *g, int32_t level, int32_t *labels, int where,
                             int32_t *n_communities);

/* Modularity Q_w (Section 2.4) of level `level`'s partition composed onto the
 * input graph (level = -1: the final partition), computed on the device as
 * the exact integer sum_C (m_w W_in(C) - Sigma_C^2) divided once, in FP64, by
 * m_w^2.  Q = 0 when m_w = 0.  Synchronous. */
slm_status slm_modularity(const slm_graph *g, int32_t level, double *q);

/* Statistics of one recorded level; level = -1 gives the last, unrecorded
 * level (the one on which the method found no more structure). */
slm_status slm_get_stats(const slm_graph *g, int32_t level, slm_level_stats *st);

/* Modularity of an arbitrary labelling (values in [0, n)) of the graph's input
 * nodes; labels in `where` memory.  Synchronous. */
slm_status slm_modularity_of(const slm_graph *g, const int32_t *labels, int where, double *q);

/* Free the graph's device memory (stream-ordered; no device-wide wait). */
void slm_destroy_graph(slm_graph *g);
/* Return the device memory cached in the library's pools (every device) to
 * the driver.  Memory still held by live handles is not affected. */
void slm_release_cached_memory(void);
const char *slm_status_string(slm_status s);
/* Message of the last error on this handle (or of the last failed create when g is NULL). */
const char *slm_last_error(const slm_graph *g);

#ifdef __cplusplus
}
#endif
#endif /* SLM_H */
