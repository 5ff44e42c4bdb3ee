/*
 * boba.h -- C ABI of libboba.so, a GB300 (sm_103a) implementation of BOBA,
 * "Batched Order By Attachment" (arXiv 2306.10410), the lightweight vertex
 * reordering of COO edge lists, plus the CSR build and SpMV used to measure
 * the locality it buys.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - A COO graph is two int32 arrays src (I) and dst (J) of length m; edge e
 *    goes src[e] -> dst[e] (Sec. 2.1).  Vertex IDs are 0-based in [0, n).
 *  - The endpoint stream is I ++ J: position i < m holds src[i], position
 *    m + e holds dst[e] (Sec. 4.3).
 *  - perm_out[k] = v means that new label k is old vertex v (p_k = v,
 *    Sec. 4.3); label = perm^-1.
 *  - Unless stated otherwise every pointer is a DEVICE pointer of the current
 *    CUDA device, owned by the caller; the library never frees or retains it.
 *    Arrays must not overlap unless an entry point says they may.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls only enqueue work: they return before the GPU finishes,
 *    and a returned BOBA_OK means the arguments were accepted and the kernels
 *    launched.  Errors found on the device (an ID outside [0, n), a spin-wait
 *    that gave up) are recorded in a per-device status word that
 *    boba_stream_status() reads; offending elements are skipped and never
 *    cause an out-of-bounds access.
 *  - Sizes above 2^31 - 1 (m, n, nnz) return BOBA_ERR_TOO_LARGE: keys are
 *    32-bit positions in [0, 2m).
 */
#ifndef BOBA_H
#define BOBA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum boba_status {
    BOBA_OK = 0,
    BOBA_ERR_INVALID_ARG = 1,      /* bad size, NULL pointer, misuse          */
    BOBA_ERR_ID_OUT_OF_RANGE = 2,  /* a vertex ID outside [0, n) was skipped  */
    BOBA_ERR_TOO_LARGE = 3,        /* m, n or nnz above 2^31 - 1              */
    BOBA_ERR_WORKSPACE = 4,        /* workspace too small / cannot grow now   */
    BOBA_ERR_TIMEOUT = 5,          /* a bounded device spin-wait gave up      */
    BOBA_ERR_CUDA = 6              /* a CUDA runtime call failed              */
} boba_status_t;

/* ------------------------------------------------------------------------
 * Reordering (Sec. 4.3 Alg. 1 and Sec. 4.4 Alg. 2 with an AtomicMin update)
 * ------------------------------------------------------------------------ */

/*
 * boba_reorder -- the BOBA ordering of one COO graph and the relabelled edges.
 *
 * Computes, for every vertex v, key(v) = the lowest position at which v occurs
 * in I ++ J (Alg. 2 with AtomicMin, Sec. 4.4, which the paper notes recovers
 * the first-occurrence order of Alg. 1, Sec. 4.3), orders the vertices that
 * occur by increasing key, and appends the vertices that occur in no edge in
 * ascending original ID.  Then rewrites each edge through the new labels
 * (Sec. 5.3): src_out[e] = label[src[e]], dst_out[e] = label[dst[e]]; edge
 * order is kept.  The result is unique and is returned bit-exactly.
 *
 *   src, dst   int32[m]   input COO (device)
 *   m          edges, 0 <= m <= 2^31 - 1
 *   n          vertices, 0 <= n <= 2^31 - 1; n = 0 requires m = 0
 *   perm_out   int32[n]   perm_out[new] = old (device)
 *   src_out    int32[m]   relabelled sources; may alias src (device)
 *   dst_out    int32[m]   relabelled destinations; may alias dst (device)
 *
 * Scratch memory comes from a workspace the library keeps per (device,
 * stream) and grows on demand with cudaMalloc; growing is refused with
 * BOBA_ERR_WORKSPACE while `stream` is being captured, so call once outside
 * capture first.  Calls on the same stream are ordered and share that
 * workspace; calls on different streams use different workspaces.
 * An ID outside [0, n) is skipped (its output element is set to -1) and
 * raises BOBA_ERR_ID_OUT_OF_RANGE in the status word.
 */
boba_status_t boba_reorder(const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                           int32_t *perm_out, int32_t *src_out, int32_t *dst_out,
                           void *stream);

/*
 * boba_reorder_workspace_bytes -- bytes of scratch boba_reorder_ex needs for
 * a graph with m edges and n vertices (0 if the sizes are invalid).
 */
size_t boba_reorder_workspace_bytes(int64_t m, int64_t n);

/*
 * boba_reorder_ex -- boba_reorder with caller-owned scratch and extra outputs.
 *
 *   label_out  int32[n] or NULL: label_out[old] = new (perm^-1)
 *   src_out, dst_out  may both be NULL: then only perm_out (and label_out)
 *              are produced -- the permutation alone, which is the figure
 *              the paper times (Sec. 1.2.4).  Giving one and not the other is
 *              BOBA_ERR_INVALID_ARG.
 *   ws         device scratch of at least boba_reorder_workspace_bytes(m, n)
 *              bytes, 256-byte aligned; contents on entry are irrelevant;
 *              must not be used by other work until this call's kernels end.
 * Never allocates; safe to capture in a CUDA graph.
 */
boba_status_t boba_reorder_ex(const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                              int32_t *perm_out, int32_t *src_out, int32_t *dst_out,
                              int32_t *label_out, void *ws, size_t ws_bytes, void *stream);

/*
 * boba_reorder_static -- boba_reorder for callers that cannot allocate device
 * memory.  (The paper has no counterpart: this is a deployment variant.)
 *
 * Who needs it: code that runs where cudaMalloc is not available or not
 * allowed -- inside a process whose device memory is all owned by one pool or
 * arena, in a plug-in whose host framework forbids allocation on its hot
 * path, or in a latency-bound loop that cannot afford the implicit device
 * synchronisation of an allocation.  Such a caller passes only its inputs and
 * outputs; the scratch lives in a fixed array inside the library's device
 * image (10 MiB, held on every GPU that loads the library until the process
 * exits).  This entry point calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *
 * Arguments and results are those of boba_reorder (same bits), plus:
 *   error_bits  device pointer to one uint32_t, or NULL.  Kernels OR
 *               (1u << code) into it for device-side errors (an ID outside
 *               [0, n): BOBA_ERR_ID_OUT_OF_RANGE; a look-back wait that gave
 *               up: BOBA_ERR_TIMEOUT); the caller clears it.  These errors are
 *               not reported by boba_stream_status().  With NULL they are not
 *               reported at all: an out-of-range ID still shows as -1 in
 *               src_out/dst_out, but a look-back wait that gave up leaves a
 *               wrong perm and wrong labels with no sign of it.  Callers that
 *               need to know pass a word.
 * With m = 0, src, dst, src_out and dst_out may be NULL (perm_out is the
 * identity).
 * Limits: m <= 2^22 edges and n <= 2^20 vertices; larger graphs return
 * BOBA_ERR_TOO_LARGE before anything is launched.
 * The first call on a device sets up that device (it looks up the device
 * address of the scratch array and caches launch sizes); make that first call
 * before any stream capture.  Every call on every stream of a device shares
 * the one scratch array, which keeps the last call's contents: calls whose
 * kernels overlap on the GPU (different streams, or other threads) race and
 * give wrong results, so order them on one stream or synchronise between
 * them.  Each call re-initialises all scratch state it relies on.
 */
boba_status_t boba_reorder_static(const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                                  int32_t *perm_out, int32_t *src_out, int32_t *dst_out,
                                  uint32_t *error_bits, void *stream);

/*
 * boba_reorder_host -- boba_reorder for a graph in HOST memory: src, dst
 * int32[m] in, perm int32[n] and src_out, dst_out int32[m] out, all HOST
 * pointers (pinned memory makes the copies asynchronous and overlapped).  The
 * edges move to the device in 2^24-edge chunks on an internal copy stream and
 * each chunk's first-occurrence pass starts as soon as it has arrived; once
 * the labels are known each chunk is relabelled and copied back on a second
 * internal stream while the next one is relabelled.  Work on `stream` before
 * the call happens before it, work after it sees the outputs.  The host
 * buffers must stay valid until then.  Calls on one device enqueue one at a
 * time (an internal lock).
 *   ws  DEVICE scratch of boba_reorder_host_workspace_bytes(m, n) bytes
 */
boba_status_t boba_reorder_host(const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                                int32_t *perm_out, int32_t *src_out, int32_t *dst_out, void *ws,
                                size_t ws_bytes, void *stream);

size_t boba_reorder_host_workspace_bytes(int64_t m, int64_t n);

/*
 * boba_reorder_variant -- boba_reorder_ex with another reading of the method:
 *   variant 0  first occurrence in I ++ J (the default; same as boba_reorder_ex)
 *   variant 1  first occurrence in the interleaved list I(0) J(0) I(1) J(1) ...,
 *              the flattening drawn in Fig. 1 (deterministic, bit-exact)
 *   variant 2  Alg. 2 exactly as printed (Sec. 4.4): a plain, racy store instead
 *              of AtomicMin, which the paper found as good in practice.  The
 *              chosen key of a vertex is one of its positions but not always the
 *              lowest, so the result may differ from run to run; it is always a
 *              valid permutation with consistent edges.
 * ws: boba_reorder_workspace_bytes(m, n) bytes.
 */
boba_status_t boba_reorder_variant(const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                                   int32_t *perm_out, int32_t *src_out, int32_t *dst_out,
                                   int variant, void *ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------
 * The reorder's phases as separate calls (sharding one graph over devices)
 * ------------------------------------------------------------------------ */

/*
 * boba_first_keys -- lowers key[v] to the lowest position of v among the
 * given edges (Alg. 2 with AtomicMin, Sec. 4.4), where local edge e holds
 * positions pos_src + e (its source) and pos_dst + e (its destination) of the
 * global stream I ++ J.  For a shard [e0, e1) of a graph with m edges, pass
 * the shard's arrays with pos_src = e0, pos_dst = m + e0.
 *   key   uint32[n] (device); init != 0 first sets every key to 0xFFFFFFFF
 * Keys of different shards combine by an elementwise MIN (all-reduce); the
 * result equals the keys of the whole graph.  Positions must stay < 2^32 - 1.
 */
boba_status_t boba_first_keys(const int32_t *src, const int32_t *dst, int64_t m_local,
                              int64_t pos_src, int64_t pos_dst, int64_t n, uint32_t *key,
                              int init, void *stream);

/* Scratch bytes for boba_labels_from_keys. */
size_t boba_labels_workspace_bytes(int64_t m_total, int64_t n);

/*
 * boba_labels_from_keys -- ParMapKeys (Alg. 2): from complete keys of a graph
 * with m_total edges, perm_out[k] = v and label_out[v] = k (label_out may be
 * NULL), vertices on no edge last in ascending ID.  key is not modified.
 */
boba_status_t boba_labels_from_keys(const uint32_t *key, int64_t m_total, int64_t n,
                                    int32_t *perm_out, int32_t *label_out, void *ws,
                                    size_t ws_bytes, void *stream);

/*
 * boba_relabel -- src_out[e] = label[src[e]], dst_out[e] = label[dst[e]]
 * (Sec. 5.3); outputs may alias inputs.  Out-of-range IDs give -1.
 */
boba_status_t boba_relabel(const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                           const int32_t *label, int32_t *src_out, int32_t *dst_out,
                           void *stream);

/* ------------------------------------------------------------------------
 * Batched reordering: G independent graphs in one persistent launch
 * ------------------------------------------------------------------------ */

/*
 * boba_reorder_batched -- BOBA (as boba_reorder) for G independent graphs
 * packed back to back, in one persistent kernel launch (after a one-block
 * planning kernel).
 *
 *   src, dst     int32[total_m] packed COO; graph g owns edges
 *                [edge_off[g], edge_off[g+1]) with LOCAL vertex IDs in
 *                [0, vert_off[g+1] - vert_off[g])                   (device)
 *   edge_off     int64[G+1], non-decreasing, edge_off[G] <= total_m   (device)
 *   vert_off     int64[G+1], non-decreasing, vert_off[G] <= total_n   (device)
 *   G            number of graphs, >= 0
 *   max_m, max_n upper bounds on any one graph's edges and vertices
 *                (<= 2^31 - 1; in the cluster mode of boba_batched_set_mode
 *                also max_n <= 442,368 = 8 x 55,296, so that a graph's key
 *                array fits in the shared memory of one 8-CTA cluster)
 *   total_m, total_n  sizes of the packed arrays (host-known)
 *   perm_out     int32[total_n], packed by vert_off, local labels    (device)
 *   src_out, dst_out int32[total_m], packed by edge_off, local labels (device)
 *   ws, ws_bytes scratch of boba_reorder_batched_workspace_bytes(G, max_m,
 *                max_n, total_m, total_n) bytes, 256-byte aligned
 *
 * Each graph's result equals boba_reorder on that graph alone, bit for bit.
 * A graph up to 55,296 vertices is reordered by one CTA in its shared memory;
 * larger ones as boba_batched_set_mode selects.  Work is claimed largest
 * graph first.  A graph whose offsets
 * are inconsistent or exceed max_m / max_n is skipped and raises
 * BOBA_ERR_INVALID_ARG in the status word.  Never allocates; safe to capture
 * in a CUDA graph.  src_out/dst_out must not alias src/dst.
 */
boba_status_t boba_reorder_batched(const int32_t *src, const int32_t *dst,
                                   const int64_t *edge_off, const int64_t *vert_off,
                                   int64_t G, int64_t max_m, int64_t max_n,
                                   int64_t total_m, int64_t total_n,
                                   int32_t *perm_out, int32_t *src_out, int32_t *dst_out,
                                   void *ws, size_t ws_bytes, void *stream);

/* Scratch bytes for boba_reorder_batched on the current device (0 if invalid). */
size_t boba_reorder_batched_workspace_bytes(int64_t G, int64_t max_m, int64_t max_n,
                                            int64_t total_m, int64_t total_n);

/*
 * boba_batched_set_mode -- how boba_reorder_batched schedules graphs above
 * 55,296 vertices.  0 = on 8-CTA clusters with the keys in distributed shared
 * memory (one persistent cluster launch for everything).  1 .. 8 = all of
 * them together, phase by phase, beside a persistent one-CTA-per-graph
 * launch for the smaller graphs; the first-occurrence and relabel phases of
 * a graph of up to S slices of 55,296 vertices keep its keys / labels in
 * shared memory, one slice per CTA, each CTA streaming all of the graph's
 * endpoints, and larger graphs use the keys in global memory.  S for the two
 * phases: 1: 8 and 1; 2: 8 and 8; 3: 8 and 2; 4: none and none; 5: 3 and
 * none; 6 (the default): as 1, except that the global-memory relabel runs
 * one CTA per SM, each claiming runs of 2^21 consecutive edges so that an
 * SM's L1 serves one graph's labels at a time; 7: as 6, with the
 * global-memory first-occurrence pass in such runs too; 8: as 7 with
 * first-occurrence S = 1.  -1 = back to the default (the autotuned choice, or
 * the BOBA_BATCH_MODE environment variable, "cluster" or "split").  All give
 * identical results.  Process-wide; host only.
 */
void boba_batched_set_mode(int mode);

/* ------------------------------------------------------------------------
 * Serving: reorder + CSR + SpMV requests under an HBM budget
 * ------------------------------------------------------------------------ */

typedef struct boba_server boba_server_t;

/*
 * boba_server_create -- a serving runtime on the current device.  Requests
 * are reordered with BOBA, converted to CSR (boba_coo_to_csr) and multiplied
 * spmv_iters times (boba_spmv_csr, y = A x with the same x), the workflow the
 * paper measures (Sec. 5.3).
 *   hbm_budget_bytes  device memory for all resident requests: allocated once
 *                     here (the only allocation of the server); requests are
 *                     admitted in arrival order while their arrays fit in it
 *   max_active        most requests on the device at once
 *   n_streams         CUDA streams the requests are spread over
 * Requests admitted together (a wave) are reordered by one batched launch;
 * each then runs on its own stream.  A request's results do not depend on
 * the other requests.  Returns NULL on invalid arguments or CUDA failure.
 */
boba_server_t *boba_server_create(size_t hbm_budget_bytes, int max_active, int spmv_iters,
                                  int n_streams);

/*
 * boba_server_submit -- enqueue a request; returns its id (>= 0), -1 for
 * invalid arguments, -2 if it could never fit in the budget.  HOST pointers:
 * src, dst int32[m]; x float[n] (NULL: x is left uninitialised); outputs
 * y float[n] and perm int32[n] (either may be NULL).  They must stay valid
 * until the request is returned by boba_server_poll; pinned memory makes the
 * copies asynchronous.
 */
int64_t boba_server_submit(boba_server_t *server, const int32_t *src, const int32_t *dst,
                           int64_t m, int64_t n, const float *x, float *y, int32_t *perm);

/*
 * boba_server_poll -- up to cap completed requests since the last poll: ids,
 * latency from submit to completion (ms), status (boba_status_t); returns the
 * number written.  After a request is returned its outputs are complete.
 */
int boba_server_poll(boba_server_t *server, int64_t *ids, double *latency_ms, int *status,
                     int cap);

/*
 * boba_server_cancel -- withdraws a request that is still waiting for
 * admission: BOBA_OK, after which the library no longer reads or writes its
 * host buffers and poll never reports it; BOBA_ERR_INVALID_ARG if the id is
 * unknown or the request has already been admitted (it then completes).
 * (A serving control; the paper has no counterpart.)
 */
boba_status_t boba_server_cancel(boba_server_t *server, int64_t id);

/* boba_server_drain -- blocks until every submitted request has completed. */
boba_status_t boba_server_drain(boba_server_t *server);

/*
 * boba_server_stats -- out[0] p50 latency (ms), out[1] p99 latency (ms),
 * out[2] throughput (Gedges/s over first arrival .. last completion),
 * out[3] requests done, out[4] edges done, out[5] peak pool bytes in use,
 * out[6] seconds spanned.  cap >= 7; returns 7.  With cap >= 13 also, and
 * returns 13: out[7] the most requests admitted at once, out[8] requests
 * admitted while others were still active (continuous batching), out[9] the
 * most requests whose device work overlapped in time (from events on their
 * streams), out[10] / out[11] p50 / p99 of the time from arrival to admission
 * (queueing, ms), out[12] p99 of the time from admission to completion
 * (service, ms).
 */
int boba_server_stats(boba_server_t *server, double *out, int cap);

/* boba_server_destroy -- drains, stops the scheduler, frees the pool. */
void boba_server_destroy(boba_server_t *server);

/* ------------------------------------------------------------------------
 * Measurement path: COO -> CSR and SpMV (Alg. 3, Sec. 1.2.2)
 * ------------------------------------------------------------------------ */

/*
 * boba_coo_to_csr -- pull CSR of a COO graph for Alg. 3: row v lists the
 * in-neighbours of v, so rows come from dst and columns from src.  Entries of
 * a row keep the input edge order (a stable sort by destination); duplicated
 * edges stay separate.  The value of the entry for edge u -> v is
 * fp32(1 / outdeg(u)), outdeg counting every edge leaving u.
 *
 *   src, dst   int32[m]             (device)
 *   row_ptr    int64[n+1]           (device)
 *   col_out    int32[m]             (device)
 *   val_out    float[m]             (device)
 *   ws         scratch of boba_coo_to_csr_workspace_bytes(m, n) bytes
 * Never allocates; safe to capture in a CUDA graph.
 */
boba_status_t boba_coo_to_csr(const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                              int64_t *row_ptr, int32_t *col_out, float *val_out,
                              void *ws, size_t ws_bytes, void *stream);

size_t boba_coo_to_csr_workspace_bytes(int64_t m, int64_t n);

/*
 * boba_spmv_csr -- y = A x for the CSR (row_ptr, col, val), Alg. 3 (pull),
 * fp32 products and fp32 accumulation.  By default rows are processed
 * warp-per-row, or several short rows per warp, in a fixed order, so the
 * result is the same run to run; rows longer than a threshold are split
 * across warps whose partial sums are combined in a fixed order through the
 * workspace.  The merge-path variant (see boba_tune_spmv) splits the work
 * evenly over row ends and nonzeros instead.
 *
 *   row_ptr int64[n_rows+1], col int32[nnz], val float[nnz] (device);
 *   x float[n_cols], y float[n_rows] (device; y must not alias x)
 *   nnz       = row_ptr[n_rows] (the host must know it)
 *   ws        scratch of boba_spmv_workspace_bytes(n_rows, nnz) bytes
 * Never allocates; safe to capture in a CUDA graph.
 */
boba_status_t boba_spmv_csr(const int64_t *row_ptr, const int32_t *col, const float *val,
                            const float *x, float *y, int64_t n_rows, int64_t nnz,
                            void *ws, size_t ws_bytes, void *stream);

size_t boba_spmv_workspace_bytes(int64_t n_rows, int64_t nnz);

/*
 * boba_pagerank -- PageRank of the graph behind a pull CSR, the PR application
 * of Sec. 5.1 (it sweeps the whole graph repeatedly until convergence).  The
 * paper fixes no constants; this is the standard power iteration with damping
 * d and the mass of vertices with no out-edge spread uniformly:
 *   pr_0(v) = 1/n,
 *   pr_{t+1}(v) = (1-d)/n + d * ( sum over entries (v,u) of val * pr_t(u)
 *                                 + (sum of pr_t(u) over u with no out-edge)/n ),
 * stopping after the first step whose L1 change sum_v |pr_{t+1}(v) - pr_t(v)|
 * is below tol, or after max_iters steps (tol = 0: exactly max_iters steps).
 * The CSR must be the one boba_coo_to_csr writes for the graph
 * (val = 1/outdeg(u), column u has an out-edge iff it occurs in col).
 * Each step is the merge-path SpMV plus one update pass; ranks are fp32,
 * the change and the dangling mass are summed in fp64 in a fixed order, so
 * the result is the same run to run.
 *
 *   row_ptr int64[n+1], col int32[nnz], val float[nnz]   (device)
 *   damping  d in [0, 1);  max_iters in [0, 2^20];  tol >= 0
 *   pr       float[n] (device): receives the ranks
 *   iters_out     int32 (device, nullable): steps taken
 *   residual_out  double (device, nullable): L1 change of the last step
 *   ws       scratch of boba_pagerank_workspace_bytes(n, nnz) bytes
 * Asynchronous: every step is enqueued at once and the steps after
 * convergence return immediately; never allocates, so it can be captured in
 * a CUDA graph.  A column ID outside [0, n) records
 * BOBA_ERR_ID_OUT_OF_RANGE and no step runs (pr stays 1/n).
 */
boba_status_t boba_pagerank(const int64_t *row_ptr, const int32_t *col, const float *val,
                            int64_t n, int64_t nnz, double damping, int64_t max_iters,
                            double tol, float *pr, int32_t *iters_out, double *residual_out,
                            void *ws, size_t ws_bytes, void *stream);

size_t boba_pagerank_workspace_bytes(int64_t n, int64_t nnz);

/*
 * boba_sort_by_dst -- reorders the edges of a COO stably by destination
 * (top_digit_only = 0: a full sort; != 0: only by the top 8 significant
 * bits of the destination as a ceil(log2 n)-bit number -- 256 bins, one
 * pass).  Sec. 5.6 suggests sorting or binning an edge
 * list that arrives in random order by destination before running BOBA;
 * sources that share a destination then sit together in I and get nearby
 * labels.  src_out/dst_out must not alias the inputs.
 *   ws  scratch of boba_sort_by_dst_workspace_bytes(m, n) bytes (device)
 */
boba_status_t boba_sort_by_dst(const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                               int32_t *src_out, int32_t *dst_out, int top_digit_only,
                               void *ws, size_t ws_bytes, void *stream);

size_t boba_sort_by_dst_workspace_bytes(int64_t m, int64_t n);

/*
 * boba_nbr -- the NBR spatial-locality metric of Sec. 5.2 over the rows of a
 * CSR: the mean, over rows with at least one entry, of
 * (distinct ids_per_line-wide lines spanned by the row's distinct column IDs)
 * / (number of distinct column IDs).  Lower is better; a row whose
 * neighbours share one line scores 1/|N(v)|.  Column IDs must be < n_rows
 * (square matrix).  Synchronous: writes the metric to *nbr_out and the number
 * of rows counted to *rows_counted (HOST pointers; the latter nullable).
 * ws: scratch of boba_nbr_workspace_bytes(n_rows, nnz) bytes (device).
 */
boba_status_t boba_nbr(const int64_t *row_ptr, const int32_t *col, int64_t n_rows, int64_t nnz,
                       int64_t ids_per_line, double *nbr_out, int64_t *rows_counted, void *ws,
                       size_t ws_bytes, void *stream);

size_t boba_nbr_workspace_bytes(int64_t n_rows, int64_t nnz);

/* ------------------------------------------------------------------------
 * Status
 * ------------------------------------------------------------------------ */

/*
 * boba_stream_status -- synchronises `stream`, then returns and clears the
 * status word of the current device: BOBA_OK, or the most severe error any
 * kernel of this library recorded on this device since the last call (the
 * word is per device, not per stream).  Returns BOBA_ERR_CUDA if the
 * synchronisation itself failed.
 */
boba_status_t boba_stream_status(void *stream);

/*
 * boba_selftest_wait_timeout -- exercises the bounded spin-wait that every
 * single-pass scan of this library uses: one warp waits for a predecessor
 * whose flag nothing ever sets, gives up after timeout_ns (1 .. 2e9), records
 * BOBA_ERR_TIMEOUT in the status word and returns, leaving the context
 * usable.  scratch: 24 bytes of device memory.  Read the result with
 * boba_stream_status().  (A diagnostic; the paper has no counterpart.)
 */
boba_status_t boba_selftest_wait_timeout(uint64_t timeout_ns, void *scratch, void *stream);

/*
 * boba_probe_gather -- a measurement aid (no step of the method): random
 * 4-byte loads at the rate this GPU sustains, the ceiling of a pass that looks
 * up one entry of an n-sized array per endpoint at a random index, as the
 * first-occurrence pass (Alg. 2, Sec. 4.4) and the relabel (Sec. 5.3) do on a
 * randomly labelled graph.  Each of a persistent grid of 256-thread blocks
 * issues loads_per_thread loads per thread at indices from a hash of a
 * per-thread counter, masked to the table.
 *   mode 0  from `table` in global memory (table_words words, read only)
 *   mode 1  from a copy of the first table_words words in each block's shared
 *           memory (table_words * 4 <= 227 KB)
 *   mode 2  from the distributed shared memory of clusters of `cluster` blocks
 *           (2, 4, 8 or 16), each block holding table_words / cluster words of
 *           the table; every load picks a block of its cluster
 *   table_words        a power of two; `table` holds at least that many words
 *   loads_per_thread   a positive multiple of 8
 *   out                uint32[out_words] (device): one sum per thread, written
 *                      so that the loads are not optimised away; the grid is
 *                      capped at out_words / 256 blocks
 *   loads_issued       HOST int64: the number of loads the launch issues
 * Asynchronous; time it with events on `stream`.  Returns
 * BOBA_ERR_INVALID_ARG for sizes outside these bounds or a cluster shape the
 * device cannot run.  (The paper has no counterpart.)
 */
boba_status_t boba_probe_gather(int mode, const uint32_t *table, int64_t table_words,
                                int64_t loads_per_thread, int cluster, uint32_t *out,
                                int64_t out_words, int64_t *loads_issued, void *stream);

/* boba_status_string -- a static, human-readable name for a status code. */
const char *boba_status_string(boba_status_t status);

/* boba_version -- a static version string of the library. */
const char *boba_version(void);

/* ------------------------------------------------------------------------
 * Autotuning (launch shapes and schedules; results never change)
 * ------------------------------------------------------------------------ */

/* Kernel families with tuned variants (the `kernel` argument below). */
enum { BOBA_TUNE_FIRST = 0, BOBA_TUNE_RELABEL = 1, BOBA_TUNE_BATCHED = 2, BOBA_TUNE_SPMV = 3,
       BOBA_TUNE_CSR = 4 };

/*
 * boba_tune_reorder -- times every variant of the first-occurrence kernel,
 * then of the relabel kernel (0..5: block size x loads in flight; 6: lanes of
 * a warp holding the same ID look it up once (warp-aggregated AtomicMin, and
 * one label gather shuffled to the group); 7: the edge streams moved between
 * global and shared memory by bulk asynchronous copies, so that only the
 * lookups go through L1), on this graph with
 * boba_reorder_ex's arguments, discards any variant whose perm/src_out/dst_out
 * differ from the default's in a single bit, and keeps the fastest for graphs
 * in the same power-of-two size class of m on this device.  chosen (int[2],
 * nullable) receives the picked variants.  Synchronous; allocates a reference
 * copy of the outputs with cudaMalloc.  Not for use during stream capture.
 */
boba_status_t boba_tune_reorder(const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                                int32_t *perm_out, int32_t *src_out, int32_t *dst_out,
                                void *ws, size_t ws_bytes, int reps, int *chosen, void *stream);

/*
 * boba_tune_batched -- the same for the schedule of boba_reorder_batched
 * (variant 0: the default split schedule, boba_batched_set_mode 6; 1: the
 * cluster mode, set_mode 0; 6: set_mode 1; 2 .. 5, 7, 8: the split schedules
 * of the same set_mode),
 * keyed by total_m.  A variant that needs more scratch than ws_bytes is
 * skipped.  An explicit boba_batched_set_mode overrides the tuned choice.
 */
boba_status_t boba_tune_batched(const int32_t *src, const int32_t *dst, const int64_t *edge_off,
                                const int64_t *vert_off, int64_t G, int64_t max_m, int64_t max_n,
                                int64_t total_m, int64_t total_n, int32_t *perm_out,
                                int32_t *src_out, int32_t *dst_out, void *ws, size_t ws_bytes,
                                int reps, int *chosen, void *stream);

/*
 * boba_tune_spmv -- the same for boba_spmv_csr (variant 0: lanes per row
 * chosen from nnz / n_rows; 1..4: 4, 8, 16, 32 lanes per row; 5..8: merge-path
 * decomposition over row ends and nonzeros with 256x8, 256x12, 512x8, 128x16
 * threads x items per tile; 9..13: merge path with a 64 KB or 32 KB cap on the
 * shared-memory carve-out, leaving the rest to L1 for the x gathers; 14:
 * 256x12 with the 64 KB cap, gathering x[0, 65536) with an L1 evict-last
 * hint: on a BOBA order the most frequent columns have the smallest
 * labels), keyed
 * by nnz.  The variants sum in different orders, so their results may differ
 * in the last bits; each is deterministic.  A variant whose y is further than
 * 1e-5 (relative L2) from variant 0's is never chosen.  Allocates a reference
 * copy of y with cudaMalloc.
 */
boba_status_t boba_tune_spmv(const int64_t *row_ptr, const int32_t *col, const float *val,
                             const float *x, float *y, int64_t n_rows, int64_t nnz, void *ws,
                             size_t ws_bytes, int reps, int *chosen, void *stream);

/*
 * boba_tune_csr -- the same for the radix passes of boba_coo_to_csr: their
 * in-tile ranking and tile shape (variant 0: 512 threads x 8 keys, eight
 * bit-ballots, registers capped for three blocks per SM, and from 2^22 keys on
 * the reduce-then-scan form of it, variant 8; 1: the same with two
 * blocks; 2: one warp match instruction; 3: per-warp shared-memory OR masks of
 * the lanes holding each digit; 4 and 5: ballots and OR masks in 256 x 16
 * tiles; 6: ballots in 384 x 16 tiles; 7: ballots in 512 x 16 tiles; 8 and
 * 9: variants 0 and 5 with the tiles' digit offsets taken from a count pass
 * and a scan of the counts instead of the look-back), keyed by m; every
 * variant's CSR must equal the default's bit for bit.
 */
boba_status_t boba_tune_csr(const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                            int64_t *row_ptr, int32_t *col_out, float *val_out, void *ws,
                            size_t ws_bytes, int reps, int *chosen, void *stream);

/* The tuned variant for a kernel family and size (0 = default), and setting it
 * by hand (variant -1 clears it). */
int boba_tune_get(int kernel, int64_t size);
void boba_tune_set(int kernel, int64_t size, int variant);

/* Persist / restore the choices of the current device (a text file, one line
 * per choice, keyed by GPU name); reset clears every choice. */
boba_status_t boba_tune_save(const char *path);
boba_status_t boba_tune_load(const char *path);
void boba_tune_reset(void);

/* ------------------------------------------------------------------------
 * Kernel timing (a measurement aid for the evaluation of Sec. 5)
 * ------------------------------------------------------------------------ */

/*
 * boba_timing_enable -- on != 0: from now on every kernel this library
 * launches is bracketed by two CUDA events recorded on the stream it is
 * launched on, and its duration is accumulated under the kernel's name.
 * Do not enable it while a stream is being captured into a CUDA graph.
 * Off by default; costs one event pair per launch when on.
 */
void boba_timing_enable(int on);

/*
 * boba_timing_collect -- waits for every recorded event pair, folds the
 * durations into per-kernel totals and returns the number of kernel names
 * seen since the last reset (or -1 on a CUDA error).
 */
int boba_timing_collect(void);

/* Name, total milliseconds and launch count of kernel record i (i < count). */
const char *boba_timing_name(int i);
double boba_timing_total_ms(int i);
int64_t boba_timing_launches(int i);

/* boba_timing_reset -- forget all totals and pending events. */
void boba_timing_reset(void);

#ifdef __cplusplus
}
#endif

#endif /* BOBA_H */
