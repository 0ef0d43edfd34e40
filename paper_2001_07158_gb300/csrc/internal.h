// internal.h -- shared declarations of the tmotif library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/tmotif.h"

namespace tmo {

typedef unsigned long long u64;
typedef unsigned int u32;

static const u32 NONE = 0xFFFFFFFFu;

// Thread-local error text behind tmotif_last_error().
void set_error(const std::string &msg);

// Status carried through the host code; the ABI returns .code.
struct Status {
    int code = TMOTIF_OK;
    bool ok() const { return code == TMOTIF_OK; }
};

Status fail(int code, const std::string &msg);
Status cuda_fail(cudaError_t e, const char *what);

#define TM_CUDA(call)                                     \
    do {                                                  \
        cudaError_t _e = (call);                          \
        if (_e != cudaSuccess) return ::tmo::cuda_fail(_e, #call); \
    } while (0)
#define TM_TRY(st)                  \
    do {                            \
        ::tmo::Status _s = (st);     \
        if (!_s.ok()) return _s;    \
    } while (0)

// Stream-ordered device memory from the library's own pool (one per device,
// memory kept cached across frees so repeated graphs and queries reuse it).
Status dev_alloc(void **p, size_t bytes, cudaStream_t s);
void dev_free(void *p, cudaStream_t s);
// Bytes a new allocation could still obtain: free device memory plus the
// pool's cached, unused blocks.
Status device_headroom(size_t *bytes);

// Colour-pair histograms are kept for up to this many colours.
static const u32 PAIR_HIST_COLORS = 64;

// A device buffer that only grows (pool memory, ordered on `stream`).
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;
    Status reserve(size_t need);
    void release();
    template <class T> T *as() const { return (T *)p; }
};

// Per-kernel-family event timing (only while profiling).
struct Profiler {
    bool on = false;
    tmotif_stats stats{};
    std::vector<cudaEvent_t> pool;
    struct Pending { cudaEvent_t a, b; int family; };
    std::vector<Pending> pending;
    size_t used = 0;
    Status begin(cudaStream_t s, cudaEvent_t *a);
    Status end(cudaStream_t s, cudaEvent_t a, int family);
    Status collect();  // after the stream is synchronised
    void destroy();
};

enum { FAM_LAYER = 0, FAM_PREP = 1, FAM_COEF = 2, FAM_OTHER = 3, FAM_STATIC = 4 };

// Bits of the per-device status word that kernels set when they meet a
// condition they cannot continue on normally; the host takes (reads and
// clears) the word after each decision and reports it as an error.
enum : u32 {
    TM_STATUS_STAGE_TIMEOUT = 1u,  // a staged layer's bulk copy did not land within its wait limit
    TM_STATUS_BOUNDS = 2u          // checked build: an index failed its bounds check (access skipped)
};
// Device bounds checks of the checked build (compiled with -DTMOTIF_CHECKED,
// libtmotif_checked.so): TM_IN(i, n, status) is true when i < n; otherwise it
// sets TM_STATUS_BOUNDS in *status and is false, and the caller skips the
// access.  It never traps.  In the normal build it is constant true.
#ifdef TMOTIF_CHECKED
__device__ __forceinline__ bool tm_in(u64 i, u64 n, u32 *status)
{
    if (i < n) return true;
    if (status) atomicOr(status, TM_STATUS_BOUNDS);
    return false;
}
#define TM_IN(i, n, status) ::tmo::tm_in((u64)(i), (u64)(n), (status))
#else
#define TM_IN(i, n, status) true
#endif
// Address of the status word on the current device.
Status status_word(u32 **p);
// Enqueue on st: move the status word (atomic exchange with 0) to *d_slot
// (device u32), then copy it to *h_slot (pinned host u32).
Status status_take_enqueue(cudaStream_t st, u32 *d_slot, u32 *h_slot);
// After the stream is synchronised: an error for a nonzero taken word.
Status status_result(u32 taken);

// Per-query scratch on the device (grown on demand, reused across queries).
struct Workspace {
    DevBuf vflag;                       // n bytes: colour in M and alive
    DevBuf slot_begin, slot_count;      // num_colors u32
    DevBuf seg_lo, seg_hi;              // n u32: filtered in-segment of each vertex
    DevBuf f_src, f_dst, f_time;        // filtered arcs (m u32 each)
    DevBuf kbits;                       // one bit per arc (whole 4096-arc tiles): kept by the filter
    DevBuf ftiles;                      // per filter tile: kept count, then exclusive offsets
    DevBuf pos;                         // m u32: last in-arc of src with time < t
    DevBuf mark;                        // m+1 u32: checkpoint flags, then indices
    DevBuf cp_in, cp_out;               // m u32
    DevBuf block_sums;                  // scan partials
    DevBuf counters;                    // small u32/u64 device scalars
    DevBuf x;                           // n * L u64: x_u^A per lane
    DevBuf C0, C1;                      // n_cp * L u64: checkpoint values
    DevBuf out;                         // L u64: per-lane sieve sums
    DevBuf wtab;                        // k * L u64: W_d^A
    DevBuf alive;                       // n bytes: extraction probe mask
    DevBuf act, act_list;               // n+1 u32 active flags/offsets, n u32 active vertices
    DevBuf arc_sum;                     // m_f u64: arc-localised sieve sums
    DevBuf partial;                     // chunks * L u64: per-chunk sieve sums
    DevBuf queue;                       // u64 team counter of the layer launches
    DevBuf rec;                         // m_f x 16 B: {dst, cp_in, cp_out, src} of the staged layer form
    DevBuf order;                       // n_chunks + 1 u32: heavy-first chunk order, then flags and offsets
    DevBuf slist;                       // n_act u32: the active vertices grouped by colour
    DevBuf gcount;                      // 2 k u32: per-colour counts and cursors of that grouping
    u32 order_chunk = 0;                // arcs per chunk the order was built for (0: none)
    void *host_pinned = nullptr;        // small pinned readback area
    size_t host_pinned_bytes = 0;
    void release();
    size_t bytes() const;
    void set_stream(cudaStream_t s);
};

// Per-graph scratch of the static preprocessing sieve (grown on demand).
struct StaticWork {
    DevBuf keep;      // pairs + 1 u32: filter flags, then offsets
    DevBuf in, out;   // filtered pair lists (owner array, then other array)
    DevBuf arrays;    // F_2..F_k, B_2..B_k, two x*B buffers: n x L u64 each
    DevBuf qv;        // n u64: per-vertex sums Q_u
    DevBuf mask;      // n bytes: kept vertices
    void set_stream(cudaStream_t s);
    void release();
};

struct Graph {
    u32 n = 0;
    u64 m_input = 0, m = 0;             // canonical arcs
    u64 self_loops = 0, duplicates = 0;
    u32 num_colors = 0;
    u32 max_time = 0;
    cudaStream_t stream = nullptr;
    // resident arcs sorted by (dst, time, src)
    u32 *d_src = nullptr, *d_dst = nullptr, *d_time = nullptr;
    u32 *d_color = nullptr;
    u32 *d_in_off = nullptr;  // n + 1: first arc of each destination's in-segment (null: m >= 2^32 - 1)
    std::shared_ptr<std::vector<u32>> h_color;  // host copy for extraction bookkeeping (ensure_host_colors)
    std::vector<u64> pair_hist;         // arcs per (colour(src), colour(dst)), if few colours
    Workspace ws;
    Profiler prof;
    size_t resident_bytes = 0;
    // static graph E_s (built on first use): s_in = [dst | src] sorted by
    // (dst, src), s_out = [src | dst] sorted by (src, dst), m_static pairs each
    bool s_built = false;
    u64 m_static = 0;
    u32 *s_in = nullptr, *s_out = nullptr;
    StaticWork sw;
    // layer-kernel launch shape per lane width, chosen by the autotuner on the
    // first decision that needs it: (arcs per team chunk, kernel variant)
    std::map<u32, std::pair<u32, u32>> layer_tune;
};

// Arc filter of a query, passed by value to the filter kernel: the time
// window and, for EC-PathMotif, the set of allowed times (n_times = 0: any).
struct ArcFilter {
    u32 t_min = 0, t_max = 0;
    u32 n_times = 0;
    u32 times[TMOTIF_KMAX];
};

struct QuerySpec {
    u32 k = 0;
    std::vector<u32> multiset;
    u32 start = TMOTIF_ANY, end = TMOTIF_ANY;
    u32 t_min = 0, t_max = 0;
    std::vector<u32> times_exact;       // EC-PathMotif tuple (empty: none)
    u64 seed = 0;
    u32 repeats = 1;
    u64 p_begin = 0, p_end = 0;         // resolved point range
    u32 flags = 0;
    ArcFilter filter() const
    {
        ArcFilter f;
        f.t_min = t_min;
        f.t_max = t_max;
        f.n_times = (u32)times_exact.size();
        for (u32 i = 0; i < f.n_times; i++) f.times[i] = times_exact[i];
        return f;
    }
};

Status parse_query(const Graph &g, const tmotif_query *q, QuerySpec *out);

// One query of a packed many-graph batch, as the device reads it (pack.cu):
// its graph's first vertex in the packed numbering, k, start/end (packed ids
// or NONE), the y key of the current repeat and the first lane-sum slot.
struct PackJob {
    u64 ky;
    u32 vbase, k, start, end;
};

// Parameters of one job's layer step (eq. gen-polynomial:3), as the layer
// kernel reads them.
struct LayerParams {
    const u32 *src, *dst, *time, *cp_in, *cp_out, *seg_hi;
    const u64 *x;
    const u64 *Cin;
    u64 *Cout;
    u64 *partial;   // last layer: per (chunk, lane) sums
    u64 *arc_sum;   // last layer, arc localisation: per filtered arc, XOR over lanes (or null)
    u64 m_f;
    u64 n_chunks;
    u64 ky;
    u32 L, lane_groups, chunk, ell, k, start, end, T;
    // packed batches only: vertex -> job, the jobs, per (job, lane) sums
    const u32 *jv = nullptr;
    const PackJob *pjobs = nullptr;
    u64 *pout = nullptr;
    // single-job launches: team counter (zeroed before the launch) from which
    // resident teams take the next team index; null: one team per team slot
    unsigned long long *queue = nullptr;
    // staged form: per filtered arc {dst, cp_in, cp_out, src} (16 bytes; the
    // times come from `time`, padded to a multiple of 4 entries)
    const uint4 *rec = nullptr;
    // the device status word (TM_STATUS_* bits), or null
    u32 *status = nullptr;
    // bounds of the checked build: vertices (x rows) and checkpoints (C rows)
    u32 n_vert = 0;
    u64 n_cp = 0;
    // staged form: bytes added to each copy's expected count (the checked
    // build's forced-timeout test; 0 otherwise)
    u32 stage_extra_tx = 0;
    // single-job launches: the order in which teams take chunks (heavy chunks
    // first), or null for index order
    const u32 *order = nullptr;
};

// One decision in flight: its query, its device workspace and its progress
// through lane batches and layers.  tmotif_decide runs one job to the end;
// the batch path and the server advance many jobs together, one shared
// layer launch per step.
struct Job {
    Graph *g = nullptr;
    QuerySpec q;
    const uint8_t *d_alive = nullptr;
    Workspace *ws = nullptr;
    cudaStream_t st = nullptr;
    Profiler *prof = nullptr;
    // sizes known after prep
    u64 mf = 0, ncp = 0, n_act = 0;
    u32 max_seg = 0;      // longest in-segment among the kept arcs
    u32 L = 0, T = 0, lane_groups = 0, chunk = 128;
    u32 variant = 0;      // layer kernel shape (see the autotuner)
    u64 n_chunks = 0;
    // progress
    u32 r = 0;            // repeat
    u64 p0 = 0;           // first point of the current lane batch
    u32 ell = 0;          // next layer to run (2..k), k+1 = batch finished
    u64 qsum = 0;
    int found = 0;
    u64 sieve_sum = 0;
    bool done = false;
    std::vector<u64> vals;  // repeat-0 per-point sums on [p_begin, p_end)
    u64 ky = 0;           // y key of the current repeat
    bool multi_slot = false;  // readouts go to per-batch host slots (one sync per decision)
    bool localize = false;    // accumulate arc-localised sums at the last layer
    u32 rep_offset = 0;       // repeat index of the first repeat this job evaluates
    u64 batch_seq = 0;    // batch number across repeats (slot index)
    bool slist_ready = false;  // the workspace's slist holds this query's active vertices by colour
};

// Job steps.  prep: filter, checkpoints, buffer sizing (synchronises the
// job's stream); batch_begin: coefficients of the lane batch at p0;
// readout_enqueue: reduce the last layer's partial sums and copy them to the
// host; readout_finish (after the stream is synchronised): accumulate and
// move on to the next batch, repeat, or finish.
Status job_prep(Job &j);
// A launch shape the autotuner found on this device for lane width L and a
// layer of about mf arcs (same floor(log2)), if any.
bool tuned_shape(u32 L, u64 mf, std::pair<u32, u32> *shape);
// Guards every graph's layer_tune map: the server's lanes prepare jobs on
// one graph from two host threads.
std::mutex &layer_tune_mutex();
// A layer launch shape the kernels accept (lane width, arcs per chunk, variant).
bool layer_shape_valid(u32 L, u32 chunk, u32 variant);
// The process-wide autotuner shapes as text, one "device L log2_arcs chunk
// variant" line each; import adds (or replaces) the lines' shapes.
std::string tuner_export();
Status tuner_import(const std::string &text);
// Checked build: the staged layer form's copies are expected to bring 16
// bytes more than they do, so that every bounded wait runs out (the test of
// the timeout path).  UNSUPPORTED in the normal build.
Status debug_stage_timeout(bool on);
// Device memory of the library's pool on the current device.
Status memory_stats(u64 *used, u64 *used_high, u64 *reserved, bool reset);
Status job_batch_begin(Job &j);
LayerParams job_layer_params(const Job &j);
Status job_readout_enqueue(Job &j);
void job_readout_finish(Job &j);
// One layer launch per lane-width class for all the given jobs (each at its
// own layer), on stream st.  `dev_params` is a device buffer for the job
// table.
Status launch_layers(cudaStream_t st, const std::vector<Job *> &jobs, DevBuf &dev_params, void *host_params,
                     size_t host_params_bytes, Profiler *prof);
// Device bytes a job will hold once prepped (for admission).
size_t job_bytes(const Job &j);
// A whole prepped job at once: job_enqueue_all enqueues every lane batch of
// every repeat (coefficients, layers, readout into a per-batch pinned slot)
// and the status word's readout on the job's stream -- with tune, layer 3 of
// the first batch runs the autotuner where the graph has no shape for the
// lane width yet; after the stream is synchronised, job_finish_all checks the
// status word and accumulates the readouts (the job is then done).
Status job_enqueue_all(Job &j, bool tune);
Status job_finish_all(Job &j);

// Decide on graph g; alive (device, n bytes, may be null) masks vertices.
// per_point (host, may be null) receives repeat-0 values on [p_begin,p_end).
Status sieve_decide(Graph &g, const QuerySpec &q, const uint8_t *d_alive, int *found, u64 *sieve_sum,
                    u64 *per_point, double *ms);

// Arcs among the vertices with alive[u] != 0 (device mask) inside the time
// window, copied to the host in (dst, time, src) order, using workspace w on
// stream st.
Status gather_arcs(Graph &g, Workspace &w, cudaStream_t st, Profiler &prof, const uint8_t *d_alive, ArcFilter f,
                   std::vector<u32> *src, std::vector<u32> *dst, std::vector<u32> *time);

// Device arrays of a graph (arcs, colours, workspace, profiler events).
void release_graph_arrays(Graph *g);
// g.h_color, copied from the device on the graph's stream at first use (the
// extraction entry points call it before their bookkeeping reads colours).
Status ensure_host_colors(Graph &g);
// The arcs of g whose endpoints both have alive[u] != 0 (device mask), as a
// new resident graph with the same vertex ids (extraction's shrinking
// subgraph).  Uses workspace w on stream st.
Status make_subgraph(const Graph &g, Workspace &w, cudaStream_t st, const uint8_t *d_alive, Graph *sub);
// Arc filter (Sec. 8.1 (i)) in two passes: _count leaves the keep mask and
// tile offsets in the workspace and the kept count in d_total (device u32);
// after the caller reads the count and sizes the outputs, _compact writes the
// kept arcs in arc order.  With in_off (the graph's in-segment offsets, n + 1
// entries) and vlist (the flagged vertices ascending, their count at device
// d_nlist) the first pass goes by vertex, else by tiles of arcs.
Status filter_arcs_count(cudaStream_t st, Workspace &w, const u32 *src, const u32 *dst, const u32 *time,
                         const u32 *in_off, u32 n, u64 m, const uint8_t *vflag, const ArcFilter &f, u32 *d_total,
                         u64 *launches, const u32 *vlist = nullptr, const u32 *d_nlist = nullptr);
// The graph's in-segment offsets d_in_off (n + 1 u32; first arc of each
// destination, arcs sorted by destination), built on st; left null when the
// arc count does not fit 32 bits.  tiles: scan scratch; d_total: a device u32.
Status build_in_off(Graph &g, cudaStream_t st, DevBuf &tiles, u32 *d_total);
Status filter_arcs_compact(cudaStream_t st, Workspace &w, const u32 *src, const u32 *dst, const u32 *time, u64 m,
                           u32 *o_src, u32 *o_dst, u32 *o_time, u64 *launches);

// Extraction (Sec. 6.9) as a state machine: next_probe() gives the next
// decision to run (the first one is the query itself, the rest mask the
// vertices with alive[u] == 0), result() takes its answer.  When
// next_probe() returns false, stage is SHRUNK (run extract_finish) or
// NOT_FOUND.
struct ExtractState {
    enum Stage { FIRST, SEARCHING, PROBING, SHRUNK, NOT_FOUND };
    struct Block { u64 lo, hi; };
    QuerySpec query;
    std::vector<uint8_t> alive;
    std::vector<u32> R;
    std::vector<Block> stack;
    u64 n_alive = 0, cur_lo = 0, cur_hi = 0, cur_cnt = 0;
    u32 probes = 0;
    Stage stage = FIRST;
    // Probes run on a compacted copy of the arcs among alive vertices, rebuilt
    // whenever the alive candidates halve (results are unchanged: masked
    // vertices contribute nothing).
    std::unique_ptr<Graph, void (*)(Graph *)> sub{nullptr, release_graph_arrays};
    u64 alive_at_build = 0;
    Graph *current(Graph &root) { return sub ? sub.get() : &root; }
    Status maybe_compact(Graph &root, Workspace &w, cudaStream_t st);
    void init(const Graph &g, const QuerySpec &q);
    bool next_probe(QuerySpec *pq);
    void result(bool yes);
    void push_halves(u64 lo, u64 hi);
};
Status extract_finish(Graph &g, Workspace &w, cudaStream_t st, Profiler &prof, const ExtractState &ex, u32 *verts,
                      u32 *times, int *found);
Status extract_path(Graph &g, const QuerySpec &q, u32 *verts, u32 *times, int *found, u32 *probes);

// The first filtered arc (lowest index) whose arc-localised sum in the job's
// workspace is nonzero; *best = NONE when there is none.  Synchronises.
Status job_first_arc(Job &j, u32 *best, u32 *a, u32 *b, u32 *t);

// Extraction by localisation as a state machine: next() gives the next
// arc-localised decision to run (its query, repeat and vertex mask),
// result() takes the first nonzero arc it found (best = NONE if none).
struct LocalizedExtract {
    QuerySpec query;
    std::shared_ptr<std::vector<u32>> color;
    std::vector<u32> ms;
    std::vector<uint8_t> alive;
    std::vector<u32> verts, times;
    u32 kk = 0, level = 0, rep = 0, cur_end = TMOTIF_ANY, cur_tmax = 0;
    u32 best = 0xFFFFFFFFu, ba = 0, bb = 0, bt = 0;
    bool done = false, found = false;
    void init(const Graph &g, const QuerySpec &q);
    bool next(QuerySpec *sub, u32 *repeat, const std::vector<uint8_t> **mask);
    void result(u32 idx, u32 a, u32 b, u32 t);
};

// Arc-localised sieve for one repeat: the job's arc sums, then the first
// filtered arc (lowest index, i.e. first in (dst, time, src) order) whose sum
// is nonzero; *best = NONE when there is none, else (*a -> *b, *t).
Status sieve_first_arc(Graph &g, const QuerySpec &q, u32 repeat, const uint8_t *d_alive, u32 *best, u32 *a, u32 *b,
                       u32 *t);
// Per-vertex localised values Q_u (Sec. 6.7) for every vertex: XOR over the
// arc sums of the arcs into u.  per_vertex (host) has n entries.
Status sieve_localize(Graph &g, const QuerySpec &q, u64 *per_vertex, int *found, u64 *sieve_sum, double *ms);
// Optimum timestamp by binary search over the window's upper end (Sec. 6.8).
Status optimum_time(Graph &g, const QuerySpec &q, u32 *t_opt, int *found);
// Extraction by localisation (k-1 arc-localised sieves, path built backwards).
Status extract_localized(Graph &g, const QuerySpec &q, u32 *verts, u32 *times, int *found);

Status build_graph(const tmotif_graph_desc *d, Graph *g);

// Packed many-graph batch (pack.cu): every query's per-point values on its
// graph, identical to deciding each alone; vals[i] receives 2^k values.
// Queries must be pack_eligible (one repeat, all points, no preprocessing).
bool pack_eligible(const QuerySpec &q);
Status pack_decide(Graph *const *graphs, const QuerySpec *specs, size_t count, cudaStream_t st,
                   std::vector<std::vector<u64>> *vals, u64 *launches);
// Stable LSD radix sort of N 64-bit keys on their low `bits` bits; a and b
// hold N keys each, *sorted points at the one with the result.
Status radix_sort_u64(cudaStream_t st, u64 *a, u64 *b, u64 N, int bits, u32 *d_scratch, u64 **sorted,
                      u64 *launches);

// Static preprocessing sieve (Sec. 8.1 (ii)): the static graph of g (built
// once), then per-vertex sums Q_u (device, n u64) for the query: nonzero iff
// u lies on a static path with colours M.  kept_pairs (optional) receives
// the number of static pairs among the query's vertices.
Status static_graph_ensure(Graph &g);
Status static_sieve(Graph &g, const QuerySpec &q, const uint8_t *d_alive, u64 *d_Qv, u64 *kept_pairs);
// d_mask[u] = (Q_u != 0), device n bytes.
Status static_mask(Graph &g, const QuerySpec &q, const uint8_t *d_alive, uint8_t *d_mask, u64 *kept_pairs);
// Device build of the resident arc arrays from the caller's host arrays:
// validation, orientation, self-loop and duplicate removal, (dst, time, src)
// order.
Status build_graph_device(const tmotif_graph_desc *d, Graph *g);
// Streaming multiprocessors of the current device (cached per device).
int sm_count();

// Device GF multiply of host arrays (diagnostic).
Status gf_mul_batch(const u64 *a, const u64 *b, u64 *out, u64 n);
// Throughput probe of the product forms (diagnostic).
Status gf_probe(int method, u32 iters, double *ms, u64 *products);

}  // namespace tmo

// The opaque ABI handle is the graph itself.
struct tmotif_graph : public tmo::Graph {};
