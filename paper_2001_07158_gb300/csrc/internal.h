// internal.h -- shared declarations of the tmotif library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

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

// A device buffer that only grows.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
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

enum { FAM_LAYER = 0, FAM_PREP = 1, FAM_COEF = 2, FAM_OTHER = 3 };

// Per-query scratch on the device (grown on demand, reused across queries).
struct Workspace {
    DevBuf vflag;                       // n bytes: colour in M and alive
    DevBuf slot_begin, slot_count;      // num_colors u32
    DevBuf seg_lo, seg_hi;              // n u32: filtered in-segment of each vertex
    DevBuf f_src, f_dst, f_time;        // filtered arcs (m u32 each)
    DevBuf keep;                        // m+1 u32: flags, then exclusive offsets
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
    void *host_pinned = nullptr;        // small pinned readback area
    size_t host_pinned_bytes = 0;
    void release();
    size_t bytes() const;
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
    std::vector<u32> h_color;           // host copy for extraction bookkeeping
    Workspace ws;
    Profiler prof;
    size_t resident_bytes = 0;
};

struct QuerySpec {
    u32 k = 0;
    std::vector<u32> multiset;
    u32 start = TMOTIF_ANY, end = TMOTIF_ANY;
    u32 t_min = 0, t_max = 0;
    u64 seed = 0;
    u32 repeats = 1;
    u64 p_begin = 0, p_end = 0;         // resolved point range
};

Status parse_query(const Graph &g, const tmotif_query *q, QuerySpec *out);

// Decide on graph g; alive (device, n bytes, may be null) masks vertices.
// per_point (host, may be null) receives repeat-0 values on [p_begin,p_end).
Status sieve_decide(Graph &g, const QuerySpec &q, const uint8_t *d_alive, int *found, u64 *sieve_sum,
                    u64 *per_point, double *ms);

// Arcs among the vertices with alive[u] != 0 (device mask) inside the time
// window, copied to the host in (dst, time, src) order.
Status gather_arcs(Graph &g, const uint8_t *d_alive, u32 t_min, u32 t_max, std::vector<u32> *src,
                   std::vector<u32> *dst, std::vector<u32> *time);

// Extraction (Sec. 5.9).
Status extract_path(Graph &g, const QuerySpec &q, u32 *verts, u32 *times, int *found, u32 *probes);

Status build_graph(const tmotif_graph_desc *d, Graph *g);

// Device GF multiply of host arrays (diagnostic).
Status gf_mul_batch(const u64 *a, const u64 *b, u64 *out, u64 n);

}  // namespace tmo

// The opaque ABI handle is the graph itself.
struct tmotif_graph : public tmo::Graph {};
