/*
 * slm_server.h -- a request server for community detection with the
 * Synchronised Louvain Method (Algorithm 1 of the paper, run per request).
 *
 * The paper describes one run on one graph; serving many graphs as they
 * arrive is a systems layer around that run, with no counterpart in the
 * paper.  A request carries one graph (symmetric CSR in HOST memory, the
 * conventions of slm_create_graph) and its options.  The server:
 *   - queues requests in arrival order;
 *   - admits the oldest waiting request as soon as a slot is free and its
 *     estimated device footprint (slm_server_footprint) fits in what is left
 *     of the HBM budget (first come, first served: a large request at the
 *     head waits for memory rather than being overtaken);
 *   - runs every admitted request on its slot's own CUDA stream, driven by
 *     its own host thread, so the device work of several requests overlaps
 *     (a request that arrives while others run starts as soon as a slot and
 *     memory free up, without waiting for the others to finish);
 *   - keeps a request's graph and label state on the device from admission
 *     to completion, then copies the final partition to host memory, frees
 *     the device state and returns its footprint to the budget.
 * A request's result depends only on its graph and options: partitions,
 * statistics and modularity are bit for bit those of slm_create_graph +
 * slm_run + slm_get_partition(-1) + slm_modularity(-1) on that graph alone.
 *
 * All functions are thread-safe.  Times are seconds on the host's monotonic
 * clock, measured from slm_server_create.  Conventions as in slm.h.
 */
#ifndef SLM_SERVER_H
#define SLM_SERVER_H

#include "slm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct slm_server slm_server; /* opaque, owned by the library */

/* One request's graph: symmetric CSR in HOST memory (row_ptr n+1 entries,
 * col_idx and weights row_ptr[n] entries; weights NULL = unit).  The server
 * copies it during slm_server_submit; the caller keeps ownership. */
typedef struct {
    int32_t n;
    const int32_t *row_ptr;
    const int32_t *col_idx;
    const int32_t *weights;
} slm_graph_desc;

/* Request states reported by slm_server_poll. */
#define SLM_REQ_QUEUED 0
#define SLM_REQ_RUNNING 1
#define SLM_REQ_DONE 2
#define SLM_REQ_FAILED 3

typedef struct {
    int32_t state;          /* SLM_REQ_* */
    int32_t status;         /* slm_status of the run (SLM_OK unless FAILED) */
    int32_t n;              /* nodes of the request's graph */
    int32_t n_communities;  /* K of the final partition (when DONE) */
    int64_t nnz;            /* stored entries of the request's graph */
    int32_t levels;         /* recorded levels of the run */
    int32_t slot;           /* slot that ran it (-1 while queued) */
    double t_submit;        /* seconds since server creation */
    double t_admit;         /* admission (slot and memory granted); 0 while queued */
    double t_done;          /* partition and modularity in host memory; 0 until then */
    double modularity;      /* final Q_w (when DONE) */
    uint64_t footprint;     /* device bytes reserved against the budget */
    uint64_t peak_bytes;    /* device bytes the run actually held at its peak */
    int64_t edges_scanned;  /* CSR entries read by the run's scans, all levels */
} slm_request_info;

typedef struct {
    int64_t submitted, completed, failed, rejected;
    int32_t queued, running;
    int32_t max_running;        /* most requests running at the same time */
    uint64_t budget_bytes;      /* the HBM budget */
    uint64_t reserved_bytes;    /* footprints of the running requests */
    uint64_t max_reserved_bytes;
} slm_server_stats;

/* Device bytes reserved for a graph of n nodes and nnz stored entries: an
 * upper bound on what one run holds at once (input CSR, per-level
 * workspace, aggregation buffers), plus a fixed allowance. */
uint64_t slm_server_footprint(int32_t n, int64_t nnz);

/* Start a server on the current device with `max_slots` slots (1..64), each
 * a host thread with its own CUDA stream, and an HBM budget in bytes.
 * Errors: INVALID_ARGUMENT, CUDA. */
slm_status slm_server_create(uint64_t hbm_budget_bytes, int32_t max_slots, slm_server **out);

/* Copy a request into the queue and return its ticket (> 0).  opt may be
 * NULL (defaults).  Errors: INVALID_ARGUMENT (bad CSR shape: the full
 * validation of slm_create_graph runs at admission and fails the request),
 * BUDGET (its footprint exceeds the whole budget: it could never be
 * admitted; nothing is queued). */
slm_status slm_server_submit(slm_server *sv, const slm_graph_desc *graph, const slm_options *opt,
                             uint64_t *ticket);

/* As slm_server_submit, with a deadline: deadline_s > 0 seconds after
 * submission the request must have ended.  A request still queued then ends
 * FAILED with SLM_ERR_DEADLINE without running (queued deadlines are checked
 * at least every 10 ms); a running one stops before its next level or sweep
 * with the same status, its device memory freed and its footprint returned.
 * deadline_s = 0: no deadline; negative or NaN: INVALID_ARGUMENT. */
slm_status slm_server_submit_deadline(slm_server *sv, const slm_graph_desc *graph,
                                      const slm_options *opt, double deadline_s, uint64_t *ticket);

/* As slm_server_submit_deadline for a directed graph: `graph` holds W as
 * out-arcs (row i lists the heads of i's arcs, sorted and unique, positive
 * weights; no symmetry required), run as slm_create_graph_directed and
 * slm_run run it (the directed Q_w of Section 2.4; the result's modularity
 * is that Q_w).  Its footprint counts U = W + W^T (at most twice the
 * entries) and the packed (out, in) strengths.  Errors as
 * slm_server_submit_deadline; what slm_create_graph_directed refuses
 * (OVERFLOW included) fails the request at admission. */
slm_status slm_server_submit_directed(slm_server *sv, const slm_graph_desc *graph,
                                      const slm_options *opt, double deadline_s, uint64_t *ticket);

/* Cancel a request.  A queued request ends FAILED with SLM_ERR_CANCELLED at
 * once (it never runs); a running one stops before its next level or sweep
 * and ends FAILED with SLM_ERR_CANCELLED (the device work already queued for
 * it finishes first; a run that completes before it looks at the flag ends
 * DONE); a request that has already ended is left as it is.  Returns SLM_OK,
 * or INVALID_ARGUMENT for an unknown or released ticket. */
slm_status slm_server_cancel(slm_server *sv, uint64_t ticket);

/* Non-blocking state of a request (SLM_REQ_*).  INVALID_ARGUMENT for an
 * unknown or released ticket. */
slm_status slm_server_poll(slm_server *sv, uint64_t ticket, int32_t *state);

/* Block until the request is DONE or FAILED, or until timeout_s seconds have
 * passed (timeout_s < 0: no limit).  Returns SLM_OK when it ended (also when
 * another thread took its result with release meanwhile), SLM_ERR_TIMEOUT
 * otherwise, INVALID_ARGUMENT for an unknown or already released ticket. */
slm_status slm_server_wait(slm_server *sv, uint64_t ticket, double timeout_s);

/* Timing and size record of a request (any state). */
slm_status slm_server_request_info(slm_server *sv, uint64_t ticket, slm_request_info *info);

/* Result of a finished request: labels (HOST, n int32, may be NULL) get the
 * final partition of its input nodes, *n_communities (may be NULL) its K,
 * *q (may be NULL) its modularity.  Returns the request's run status
 * (SLM_OK when DONE); NOT_RUN while it is queued or running.  With
 * release != 0 the ticket and its memory are dropped afterwards. */
slm_status slm_server_result(slm_server *sv, uint64_t ticket, int32_t *labels,
                             int32_t *n_communities, double *q, int32_t release);

slm_status slm_server_get_stats(slm_server *sv, slm_server_stats *st);

/* Stop accepting requests, drop the queued ones (they end FAILED with
 * SLM_ERR_NOT_RUN), wait for the running ones and free everything.  Threads
 * blocked in slm_server_wait on this server return once their request has
 * ended, and destroy frees nothing before they have left.  No other call on
 * the same server may start once destroy has begun. */
void slm_server_destroy(slm_server *sv);

/* Message of the last error of the server (or of the last failed create when sv is NULL). */
const char *slm_server_last_error(const slm_server *sv);

#ifdef __cplusplus
}
#endif
#endif /* SLM_SERVER_H */
