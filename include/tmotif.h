/*
 * tmotif.h -- C ABI of the GB300 temporal path-motif sieve.
 *
 * The library decides PathMotif (Sec. 5.3 of Thejaswi, Gionis, Lauri, "Finding
 * path motifs in large temporal graphs using algebraic fingerprints"): given a
 * vertex-coloured temporal graph and a multiset M of k colours, is there a
 * temporal path (k distinct vertices, arcs with strictly increasing
 * timestamps, Sec. 4) whose vertex colours are exactly M?  It evaluates the
 * constrained multilinear sieve of Lemma 6.5 over GF(2^64): the temporal-walk
 * generating function of eq. (gen-polynomial:3) at 2^k sieve points, summed;
 * a nonzero sum certifies a matching path.  Extraction follows Sec. 6.9 (self-
 * reducibility with halving, then temporal DFS).
 *
 * Conventions (all entry points):
 *   - Every call returns TMOTIF_OK (0) or a TMOTIF_ERR_* code and never aborts
 *     the process; tmotif_last_error() gives a message for the calling thread.
 *   - Pointers in descriptors are HOST pointers owned by the caller; the
 *     library copies what it keeps.  Outputs go to caller-owned host buffers.
 *   - Handles are owned by the library and released by the matching destroy.
 *   - Vertex ids are in [0, n).  Timestamps are >= 1 (Z_+, Sec. 4).
 *   - 2 <= k <= TMOTIF_KMAX.  Colours are in [0, num_colors).
 *   - A YES answer (found = 1) is always right: the sieve's error is one-sided
 *     (Lemmas 6.3/6.5).  A NO is wrong with probability at most
 *     (2k-1)/2^64 per independent repeat (Sec. 6.5).
 *   - Work runs on the CUDA stream given at graph creation (NULL = the legacy
 *     default stream); calls return after their results are on the host.
 *   - A graph handle is used by one thread at a time.
 */
#ifndef TMOTIF_H
#define TMOTIF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TMOTIF_ANY 0xFFFFFFFFu
#define TMOTIF_KMAX 20
/* tmotif_query.flags: extract by halving self-reduction + DFS instead of by
 * localisation (see tmotif_extract). */
#define TMOTIF_EXTRACT_HALVING 1u
/* tmotif_query.flags: extract an optimum solution -- a path whose latest arc
 * time is the least possible (tmotif_optimum_time), as in Sec. 6.8-6.9. */
#define TMOTIF_EXTRACT_OPTIMUM 2u
/* tmotif_query.flags: static preprocessing sieve first (Sec. 8.1 (ii); see
 * tmotif_static_sieve): decide / extract / optimum time / localise on the
 * temporal graph restricted to the vertices it keeps.  Every temporal match
 * survives, so decisions are unchanged; per-point sums are those of the
 * restricted graph.  Not accepted by tmotif_decide_batch or tmotif_submit
 * (UNSUPPORTED). */
#define TMOTIF_PREPROCESS_STATIC 4u

enum {
    TMOTIF_OK = 0,
    TMOTIF_ERR_INVALID = 1,     /* malformed argument or graph              */
    TMOTIF_ERR_OOM = 2,         /* device or host allocation failed         */
    TMOTIF_ERR_CUDA = 3,        /* a CUDA call failed                       */
    TMOTIF_ERR_TIMEOUT = 4,     /* a bounded device or host wait gave up    */
    TMOTIF_ERR_UNSUPPORTED = 5, /* outside the supported range (e.g. k = 1) */
    TMOTIF_ERR_NOT_FOUND = 6,   /* unknown ticket                           */
    TMOTIF_ERR_BUSY = 7,        /* over the admission budget; retry later   */
    TMOTIF_ERR_CANCELLED = 8    /* the request was cancelled (tmotif_cancel) */
};

typedef struct tmotif_graph *tmotif_graph_t;   /* opaque, library-owned */
typedef struct tmotif_server *tmotif_server_t; /* opaque, library-owned */

/* A vertex-coloured temporal graph G^tau = (V, E^tau), Sec. 4.  Edge e is the
 * triple (src[e], dst[e], time[e]); with undirected = 0 it is the arc
 * src -> dst (moving from src to dst at that time); with undirected = 1 it
 * stands for both arcs.  E^tau is a set: identical arcs are kept once and
 * self-loops are dropped (tmotif_graph_info reports both counts).  Arrays are
 * caller-owned host memory of m (edges) and n (colours) entries. */
typedef struct {
    uint32_t n;
    uint64_t m;
    const uint32_t *src, *dst, *time;
    const uint32_t *color;
    uint32_t num_colors;
    uint32_t undirected;
    void *cuda_stream; /* cudaStream_t used for every call on this graph */
} tmotif_graph_desc;

/* A PathMotif query (Sec. 5.3), with the (s,d) variant of Sec. 7.1 as start/
 * end vertices and the latest-time restriction of Sec. 6.8 as a window.
 *   multiset      k colours in any order (caller-owned host array);
 *   start, end    TMOTIF_ANY or the required first / last vertex; M must count
 *                 their colours;
 *   t_min, t_max  only arcs with t_min <= time <= t_max are used (t_max = 0:
 *                 no upper bound);
 *   seed          selects the random evaluation point; repeats >= 1
 *                 independent evaluations, found = OR over them;
 *   point_begin, point_end  0,0 = all 2^k sieve points; otherwise only the
 *                 points [point_begin, point_end) are evaluated (sharding a
 *                 query across devices; combine the per-point sums by XOR);
 *   flags         0 or TMOTIF_EXTRACT_HALVING, TMOTIF_EXTRACT_OPTIMUM and/or
 *                 TMOTIF_PREPROCESS_STATIC;
 *   timestamps    NULL, or the EC-PathMotif tuple T = (j_1, ..., j_{k-1}) of
 *                 Sec. 7.3 (caller-owned host array of k-1 strictly increasing
 *                 times >= 1; INVALID otherwise): the path's l-th arc must have
 *                 time j_l.  Only arcs whose time is in T (and in the window)
 *                 are used; a temporal path of k-1 arcs with strictly
 *                 increasing times from a set of k-1 values uses them all in
 *                 order, so this is exactly the EC recurrence of Sec. 7.3.
 *                 Applies to decide, extract, batch and server requests. */
typedef struct {
    uint32_t k;
    const uint32_t *multiset;
    uint32_t start, end;
    uint32_t t_min, t_max;
    uint64_t seed;
    uint32_t repeats;
    uint32_t point_begin, point_end;
    uint32_t flags;
    const uint32_t *timestamps;
} tmotif_query;

/* Result of tmotif_decide.  per_point is caller-owned and optional (NULL or
 * room for point_end - point_begin values, 2^k when both are 0); it receives
 * the sieve sums Q^A of the first repeat, point p <-> A = {j : bit j of p}.
 * sieve_sum is their XOR; ms is the device time of the call. */
typedef struct {
    int found;
    uint64_t sieve_sum;
    uint64_t *per_point;
    double ms;
} tmotif_decision;

typedef struct {
    uint32_t n;
    uint64_t m_input;     /* edges passed in                               */
    uint64_t m_arcs;      /* canonical arcs kept on the device              */
    uint64_t self_loops;  /* dropped                                        */
    uint64_t duplicates;  /* identical arcs merged                          */
    uint32_t max_time;
    uint64_t device_bytes;/* resident graph plus current workspace         */
} tmotif_graph_info;

/* Cumulative device time per kernel family (CUDA events on the graph's
 * stream), recorded only while profiling is on.  bytes_* count the
 * algorithmic traffic the layer kernels were asked to move. */
typedef struct {
    uint64_t launches;         /* every kernel this library launched        */
    uint64_t layer_launches;
    double layer_ms;           /* generating-function layers (eq. 3)        */
    double prep_ms;            /* per-query filter, segments, checkpoints   */
    double coef_ms;            /* sieve coefficients x_u^A (eq. motif:1)    */
    double other_ms;
    uint64_t layer_arc_lanes;  /* arcs x lanes processed by layer kernels   */
    uint64_t layer_cp_lanes;   /* checkpoints x lanes written               */
    uint64_t layer_bytes;      /* algorithmic bytes of the layer kernels    */
    uint64_t layer_gf_muls;    /* GF(2^64) products in the layer kernels    */
    uint64_t layer_table_muls; /* ... of which by a shared multiplier table  */
    uint64_t layer_table_builds; /* shared tables built (one per arc and table layer) */
    uint64_t static_launches;  /* static preprocessing sieve layers (Sec. 8.1 (ii)) */
    double static_ms;
    uint64_t static_gf_muls;   /* GF(2^64) products in those layers           */
    uint64_t static_table_muls;  /* ... of which by a shared multiplier table */
    uint64_t static_table_builds;
} tmotif_stats;

/* Build the resident graph: validate, orient, drop self-loops, merge
 * duplicates, sort arcs by (dst, time, src) and upload.  Errors: INVALID for
 * an id >= n, time 0 or colour >= num_colors; OOM; CUDA. */
int tmotif_create_graph(const tmotif_graph_desc *desc, tmotif_graph_t *out);
void tmotif_destroy_graph(tmotif_graph_t g);
int tmotif_graph_get_info(tmotif_graph_t g, tmotif_graph_info *info);

/* Decide PathMotif (Lemma 6.5 on eq. gen-polynomial:3, Lemma 6.4 time and
 * O(m L) space per lane batch of L points).  Errors: INVALID (bad multiset
 * colour, start/end out of range, repeats 0, bad point range), UNSUPPORTED
 * (k outside [2, TMOTIF_KMAX]), OOM, CUDA. */
int tmotif_decide(tmotif_graph_t g, const tmotif_query *q, tmotif_decision *out);

/* Extract one matching temporal path (Sec. 6.9): verts receives k vertex ids
 * in path order and times the k-1 arc timestamps (caller-owned).  found = 0
 * when no path exists.  Two procedures, both deterministic given the seed:
 *   by localisation (default; the paper's second approach, with the sieve of
 *     Sec. 6.7 localised to arcs): level 1 runs the sieve of the query with
 *     per-arc sums at the last layer and takes the first arc (a1 -> b1, t1)
 *     in (dst, time, src) order whose sum is nonzero -- a matching path ends
 *     with it; level j asks for a path on the remaining colours ending at
 *     a_{j-1} with all times below t_{j-1} and the later vertices masked, and
 *     takes its first nonzero arc into a_{j-1}; k-1 sieves of shrinking size.
 *     Level j uses seed mix(seed ^ j * 0xD1B54A32D192ED03);
 *   by halving (flags = TMOTIF_EXTRACT_HALVING; the paper's first approach):
 *     candidates (vertices whose colour is in M) in ascending id; a block of
 *     candidates is removed when the query stays YES without it, otherwise it
 *     is halved; probe i uses seed mix(seed ^ i * 0xD1B54A32D192ED03); the
 *     survivors go to a temporal DFS over start vertices in ascending id and
 *     arcs in (time, dst) order.
 * Errors as tmotif_decide. */
int tmotif_extract(tmotif_graph_t g, const tmotif_query *q, uint32_t *verts, uint32_t *times, int *found);

/* Optimum timestamp (Sec. 6.8): *t_opt = the least t' such that the query
 * restricted to arcs with t_min <= time <= t' is YES, found by binary search
 * with O(log t) decisions (each with the query's seed and repeats):
 * lo = max(t_min, 1), hi = t_max (0: the largest time); no path when hi is
 * NO; otherwise mid = lo + (hi - lo) / 2 moves hi to mid on YES and lo to
 * mid + 1 on NO.  *found = 0 when no path exists.  Errors as tmotif_decide. */
int tmotif_optimum_time(tmotif_graph_t g, const tmotif_query *q, uint32_t *t_opt, int *found);

/* Vertex-localised sieve (Sec. 6.7): per_vertex[u] (caller-owned, n values)
 * receives Q_u = sum over the 2^k points of P_{u,k,t}(z^A) -- nonzero exactly
 * when (w.h.p.) a matching temporal path ends at u; out receives the whole
 * decision (first repeat; repeats are ignored).  Errors as tmotif_decide. */
int tmotif_localize(tmotif_graph_t g, const tmotif_query *q, uint64_t *per_vertex, tmotif_decision *out);

/* Static preprocessing sieve (Sec. 8.1 (ii), static generating function
 * eq. gen-polynomial:1).  The temporal arcs are merged into the static graph
 * E_s = {(a, b) : some arc a -> b}; per_vertex[u] (caller-owned, n values, or
 * NULL) receives Q_u = sum over the 2^k points A of
 *   sum_{r=1..k} F_r(u) B_{k-r+1}(u),
 *   F_1(u) = x_u [u start-ok], F_l(u) = x_u sum_{(v,u)} yf(v->u, l-1) F_{l-1}(v),
 *   B_1(u) = [u end-ok],      B_l(u) = sum_{(u,w)} yb(u->w, k-l+1) x_w B_{l-1}(w),
 * with yf(a->b, p) = mix64(mix64(kf ^ (a << 32 | b)) ^ p), yb likewise with
 * kb, kf = mix64(qs ^ 0x4444444444444444), kb = mix64(qs ^ 0x5555555555555555)
 * and qs the repeat-0 query seed: nonzero exactly when (w.h.p.) u lies on a
 * static path with colours M (start/end as given).  kept (optional)
 * receives the number of such vertices.  The time window and EC timestamps
 * do not restrict E_s.  Errors as tmotif_decide. */
int tmotif_static_sieve(tmotif_graph_t g, const tmotif_query *q, uint64_t *per_vertex, uint32_t *kept);

/* Decide many (graph, query) pairs in one pass: every query runs its sieve
 * and the per-query phases of all of them share persistent launches (the
 * batched form for many small graphs).  out has count entries.  Graphs must
 * share one CUDA stream.  Errors as tmotif_decide; on error no result is
 * valid. */
int tmotif_decide_batch(const tmotif_graph_t *graphs, const tmotif_query *queries, uint32_t count,
                        tmotif_decision *out);

/* Serving: a request loop that admits decide/extract requests against
 * resident graphs while the device memory they need fits hbm_budget_bytes,
 * runs admitted requests concurrently on the device and completes them
 * asynchronously.  tmotif_submit copies the query and returns a ticket at
 * once (BUSY if the request alone exceeds the budget); tmotif_poll reports
 * done = 1 with the result once finished (verts/times may be NULL for
 * decide requests; they need room for k and k-1 entries otherwise).  For a
 * decide request, out->per_point (caller-owned, optional: NULL or room for
 * point_end - point_begin values, 2^k when both are 0) receives the same
 * per-point sums tmotif_decide gives; extract requests leave it untouched.
 * A finished ticket is forgotten after it is polled.
 * Requests run in two lanes that share the memory budget, each with its own
 * host worker thread and CUDA streams: requests over about 4e9 arc-lane steps
 * (kept arcs x (k-1) x points, doubled for extraction) run one at a time in
 * arrival order on streams of the device's greatest priority; smaller ones
 * run together, in shared layer launches, on streams of its least priority,
 * beside the large one.  Results never depend on the lane or the mix. */
int tmotif_server_create(size_t hbm_budget_bytes, tmotif_server_t *out);
int tmotif_submit(tmotif_server_t s, tmotif_graph_t g, const tmotif_query *q, int is_extract, uint64_t *ticket);
int tmotif_poll(tmotif_server_t s, uint64_t ticket, tmotif_decision *out, uint32_t *verts, uint32_t *times,
                int *done);
/* Blocking form of tmotif_poll: waits at most timeout_ms for the request to
 * finish.  TIMEOUT when it has not (the request stays pending and can be
 * polled or waited for again); otherwise as tmotif_poll with done = 1. */
int tmotif_wait(tmotif_server_t s, uint64_t ticket, uint32_t timeout_ms, tmotif_decision *out, uint32_t *verts,
                uint32_t *times);
/* Cancel a request.  One not yet admitted is dropped; one whose decisions are
 * running stops after its current decision (a decision already on the
 * device is not interrupted).  Either way it then completes with
 * TMOTIF_ERR_CANCELLED, which tmotif_poll / tmotif_wait report once (then
 * the ticket is forgotten).  A request that had already finished keeps its
 * result.  NOT_FOUND for an unknown ticket. */
int tmotif_cancel(tmotif_server_t s, uint64_t ticket);
void tmotif_server_destroy(tmotif_server_t s);

/* Profiling counters for a graph (see tmotif_stats).  set_profiling(g, 1)
 * enables per-kernel events and clears the counters. */
int tmotif_set_profiling(tmotif_graph_t g, int on);

/* Launch shape of the generating-function layer kernel for lane width L (a
 * power of two in [4, 128]) on graph g: arcs per team chunk (64, 128, 256,
 * 512 or 1024)
 * and the kernel variant (0 = the default form; 1 = at most 64 registers per
 * thread, 2 = at most 128, for L = 16 and 64; 3 = 16-thread teams at 2 lanes
 * per thread instead of the default warp team at one lane, for L = 32; 1 =
 * two 64-lane teams per chunk at 2 lanes per thread instead of one warp at 4,
 * for L = 128; 4 = the staged form for L = 32, 64 and 128: the default warp
 * team, with each team's arc metadata copied into shared memory by 1-D bulk
 * copies, cp.async.bulk, and read back as broadcasts instead of shuffles).
 * The library's autotuner picks it on the first decision that
 * needs it, by timing every candidate on one layer; set pins it (results
 * never depend on it), get reads it (NOT_FOUND when none is set yet).
 * Errors: INVALID for a bad L, chunk or variant. */
int tmotif_set_layer_shape(tmotif_graph_t g, uint32_t L, uint32_t chunk, uint32_t variant);
int tmotif_get_layer_shape(tmotif_graph_t g, uint32_t L, uint32_t *chunk, uint32_t *variant);
int tmotif_get_stats(tmotif_graph_t g, tmotif_stats *out);

/* Diagnostic: out[i] = a[i] * b[i] in GF(2^64) computed by the device
 * multiply of the sieve kernels (host arrays of n entries). */
int tmotif_gf_mul_batch(const uint64_t *a, const uint64_t *b, uint64_t *out, uint64_t n);

/* Diagnostic throughput probe of the two GF(2^64) product forms the layer
 * kernel uses, on register-resident data (no memory traffic), 8 blocks of 256
 * threads per SM: method 0 = register multiply (Karatsuba over 32x32
 * carry-less products with holes); method 1 = a warp builds the 16 x 16 nibble
 * table of one multiplier in shared memory and applies it to 64 lanes (2 per
 * thread); method 2 = the same table applied to 128 lanes (4 per thread).
 * Runs `iters` rounds; ms receives the device time, products the products
 * done.  INVALID for another method or iters = 0. */
int tmotif_gf_probe(int method, uint32_t iters, double *ms, uint64_t *products);

/* Decision without any memory allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory when they
 * need an answer -- a host program whose own allocator already holds the whole
 * device, a latency-bound loop where cudaMalloc/cudaFree would synchronise the
 * device, or code living under a memory budget fixed elsewhere.  It computes
 * the same per-point sieve sums as tmotif_decide (first repeat only) and
 * allocates nothing: every intermediate lives in one fixed device array of
 * TMOTIF_NOALLOC_SCRATCH_BYTES that each GPU loading the library keeps until
 * the process exits.
 *   d_src, d_dst, d_time  caller-owned DEVICE arrays of m canonical arcs
 *                 (ids < n, time >= 1, no self-loops, no duplicates) sorted
 *                 strictly by (dst, time, src) -- the resident layout of a
 *                 graph built by tmotif_create_graph;
 *   d_color       caller-owned DEVICE array of n colours < num_colors;
 *   q             as for tmotif_decide, with repeats == 1;
 *   d_per_point   caller-owned DEVICE output of point_end - point_begin
 *                 values (2^k when both are 0); XOR them for the sieve sum;
 *   cuda_stream   stream for all work; the call returns after it finished.
 * A graph without arcs (m = 0) gives all-zero sums.
 * Errors: UNSUPPORTED when the graph needs more scratch than the fixed array
 * (the message gives both sizes) or k is outside [2, TMOTIF_KMAX]; INVALID for
 * arcs that are not canonical and sorted, m >= 2^32 - 1, a vertex colour (of
 * any vertex, with or without arcs) >= num_colors, or bad query fields; CUDA.
 * All calls share the array and it keeps the previous call's contents; each
 * call clears what must start at zero.  Calls whose work overlaps on the GPU
 * (other streams or host threads on the same device) race on the array and
 * must be serialised by the caller.  Every call synchronises cuda_stream
 * before it returns.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  The address is kept for the life of
 * the process: after a cudaDeviceReset of a device, do not call this entry
 * point on that device again. */
#define TMOTIF_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int tmotif_decide_noalloc(const uint32_t *d_src, const uint32_t *d_dst, const uint32_t *d_time, uint64_t m,
                          const uint32_t *d_color, uint32_t n, uint32_t num_colors, const tmotif_query *q,
                          uint64_t *d_per_point, void *cuda_stream);

/* Device memory of the library's stream-ordered pool on the current device
 * (graphs, workspaces and server jobs all draw on it): bytes in use now, the
 * most in use since the last reset, and bytes the pool holds from the device
 * (freed blocks stay cached for reuse).  Any pointer may be NULL; reset = 1
 * restarts the high-water mark.  Errors: CUDA. */
int tmotif_memory_stats(uint64_t *used, uint64_t *used_high, uint64_t *reserved, int reset);

/* The autotuner's launch shapes for the whole process (per device, lane width
 * and layer size class; see tmotif_set_layer_shape), as text: one line
 * "device L log2_arcs chunk variant" per shape, so that a later process can
 * start from them instead of tuning again.
 *   export: writes at most cap - 1 bytes of the text and a NUL to buf (cap =
 *   0: nothing written) and the text's full length to *len;
 *   import: adds the lines' shapes, replacing those with the same key;
 *   blank lines are skipped.  INVALID for a malformed line or a shape the
 *   kernels do not accept; nothing is added then. */
int tmotif_tuner_export(char *buf, size_t cap, size_t *len);
int tmotif_tuner_import(const char *text);

/* 1 for the checked build (libtmotif_checked.so, compiled with
 * -DTMOTIF_CHECKED), 0 otherwise.  The checked build tests, on the device,
 * the indices the kernels derive from their inputs (vertex ids of arcs, in-
 * segment offsets, checkpoint numbers, lane indices, colour slots) before each
 * access; a failed test skips the access and sets a status bit, and the call
 * that ran the kernel returns TMOTIF_ERR_INVALID.  No check traps.  Every call
 * of both builds reads the status word after its work (a failed staged bulk
 * copy wait gives TMOTIF_ERR_TIMEOUT). */
uint32_t tmotif_checked_build(void);

/* Checked build only (UNSUPPORTED otherwise): on = 1 makes every later
 * staged layer launch (tmotif_set_layer_shape variant 4) expect 16 bytes more
 * than its bulk copies bring, so each of its bounded waits (0.1 s in this
 * build) runs out: the copies land and nothing stays in flight, the teams
 * finish from global memory, and the call reports TMOTIF_ERR_TIMEOUT.  This
 * is the test of the timeout path; on = 0 restores normal launches. */
int tmotif_debug_stage_timeout(int on);

/* Message for the last error on the calling thread (never NULL). */
const char *tmotif_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TMOTIF_H */
