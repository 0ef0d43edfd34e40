// api.cu -- the extern "C" entry points of include/tmotif.h, error handling,
// device buffers, profiling and graph residency.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "gf64.cuh"
#include "internal.h"

namespace tmo {

static thread_local std::string g_last_error = "no error";

void set_error(const std::string &msg) { g_last_error = msg; }

Status fail(int code, const std::string &msg)
{
    set_error(msg);
    Status s;
    s.code = code;
    return s;
}

Status cuda_fail(cudaError_t e, const char *what)
{
    std::string msg = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
    int code = (e == cudaErrorMemoryAllocation) ? TMOTIF_ERR_OOM : TMOTIF_ERR_CUDA;
    cudaGetLastError();  // clear sticky-free errors so later calls can proceed
    return fail(code, msg);
}

static std::mutex g_pool_mutex;
static cudaMemPool_t g_pools[256];

static Status pool_for_current_device(cudaMemPool_t *out)
{
    int dev = 0;
    TM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return fail(TMOTIF_ERR_UNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool;
        TM_CUDA(cudaMemPoolCreate(&pool, &props));
        unsigned long long keep = ~0ull;  // keep freed memory cached in the pool
        TM_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
        g_pools[dev] = pool;
    }
    *out = g_pools[dev];
    return Status();
}

Status dev_alloc(void **p, size_t bytes, cudaStream_t s)
{
    *p = nullptr;
    cudaMemPool_t pool = nullptr;
    TM_TRY(pool_for_current_device(&pool));
    cudaError_t e = cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 256), pool, s);
    if (e == cudaErrorMemoryAllocation) {
        // the pool keeps freed blocks cached; hand them back to the device
        // (after every pending free has happened) and try once more
        cudaGetLastError();
        cudaDeviceSynchronize();
        cudaMemPoolTrimTo(pool, 0);
        e = cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 256), pool, s);
    }
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, "device allocation");
    }
    return Status();
}

Status device_headroom(size_t *bytes)
{
    *bytes = 0;
    cudaMemPool_t pool = nullptr;
    TM_TRY(pool_for_current_device(&pool));
    size_t free_b = 0, total_b = 0;
    TM_CUDA(cudaMemGetInfo(&free_b, &total_b));
    unsigned long long reserved = 0, used = 0;
    TM_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved));
    TM_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
    *bytes = free_b + (size_t)(reserved > used ? reserved - used : 0);
    return Status();
}

bool layer_shape_valid(u32 L, u32 chunk, u32 variant)
{
    const bool pow2 = L >= 4 && L <= 128 && (L & (L - 1)) == 0;
    const bool ch = chunk == 64 || chunk == 128 || chunk == 256 || chunk == 512 || chunk == 1024;
    const bool var = variant == 0 || (variant <= 2 && (L == 16 || L == 64)) || (variant == 3 && L == 32) ||
                     (variant == 1 && L == 128) || (variant == 4 && (L == 32 || L == 64 || L == 128));
    return pow2 && ch && var;
}

Status memory_stats(u64 *used, u64 *used_high, u64 *reserved, bool reset)
{
    cudaMemPool_t pool = nullptr;
    TM_TRY(pool_for_current_device(&pool));
    unsigned long long u = 0, h = 0, r = 0;
    TM_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &u));
    TM_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &h));
    TM_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &r));
    if (used) *used = u;
    if (used_high) *used_high = h;
    if (reserved) *reserved = r;
    if (reset) {
        unsigned long long zero = 0;  // the high-water mark restarts from the current use
        TM_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero));
    }
    return Status();
}

void dev_free(void *p, cudaStream_t s)
{
    if (p) cudaFreeAsync(p, s);
}

Status DevBuf::reserve(size_t need)
{
    if (need <= bytes && p) return Status();
    release();
    size_t want = std::max<size_t>(need, 256);
    TM_TRY(dev_alloc(&p, want, stream));
    bytes = want;
    return Status();
}

int sm_count()
{
    static int counts[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (!counts[dev]) {
        int c = 0;
        if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c <= 0) return 1;
        counts[dev] = c;
    }
    return counts[dev];
}

void DevBuf::release()
{
    dev_free(p, stream);
    p = nullptr;
    bytes = 0;
}

void Workspace::set_stream(cudaStream_t s)
{
    DevBuf *all[] = {&vflag, &slot_begin, &slot_count, &seg_lo, &seg_hi, &f_src, &f_dst, &f_time, &kbits, &ftiles, &pos,
                     &mark, &cp_in, &cp_out, &block_sums, &counters, &x, &C0, &C1, &out, &wtab, &alive, &partial, &act, &act_list,
                     &arc_sum, &queue, &rec, &order, &slist, &gcount};
    for (DevBuf *b : all) b->stream = s;
}

void Workspace::release()
{
    DevBuf *all[] = {&vflag, &slot_begin, &slot_count, &seg_lo, &seg_hi, &f_src, &f_dst, &f_time, &kbits, &ftiles, &pos,
                     &mark, &cp_in, &cp_out, &block_sums, &counters, &x, &C0, &C1, &out, &wtab, &alive, &partial, &act, &act_list,
                     &arc_sum, &queue, &rec, &order, &slist, &gcount};
    for (DevBuf *b : all) b->release();
    if (host_pinned) cudaFreeHost(host_pinned);
    host_pinned = nullptr;
    host_pinned_bytes = 0;
}

size_t Workspace::bytes() const
{
    const DevBuf *all[] = {&vflag, &slot_begin, &slot_count, &seg_lo, &seg_hi, &f_src, &f_dst, &f_time, &kbits, &ftiles, &pos,
                           &mark, &cp_in, &cp_out, &block_sums, &counters, &x, &C0, &C1, &out, &wtab, &alive, &partial, &act, &act_list,
                           &arc_sum, &queue, &rec, &order, &slist, &gcount};
    size_t s = 0;
    for (const DevBuf *b : all) s += b->bytes;
    return s;
}

// ---------------------------------------------------------------------------
// Profiler
// ---------------------------------------------------------------------------
Status Profiler::begin(cudaStream_t s, cudaEvent_t *a)
{
    *a = nullptr;
    if (!on) return Status();
    if (used + 2 > pool.size()) {
        for (int i = 0; i < 16; i++) {
            cudaEvent_t e;
            TM_CUDA(cudaEventCreate(&e));
            pool.push_back(e);
        }
    }
    *a = pool[used++];
    TM_CUDA(cudaEventRecord(*a, s));
    return Status();
}

Status Profiler::end(cudaStream_t s, cudaEvent_t a, int family)
{
    if (!on || !a) return Status();
    cudaEvent_t b = pool[used++];
    TM_CUDA(cudaEventRecord(b, s));
    pending.push_back({a, b, family});
    return Status();
}

Status Profiler::collect()
{
    if (!on) return Status();
    for (const Pending &p : pending) {
        TM_CUDA(cudaEventSynchronize(p.b));
        float ms = 0;
        TM_CUDA(cudaEventElapsedTime(&ms, p.a, p.b));
        if (p.family == FAM_LAYER) stats.layer_ms += ms;
        else if (p.family == FAM_PREP) stats.prep_ms += ms;
        else if (p.family == FAM_COEF) stats.coef_ms += ms;
        else if (p.family == FAM_STATIC) stats.static_ms += ms;
        else stats.other_ms += ms;
    }
    pending.clear();
    used = 0;
    return Status();
}

void Profiler::destroy()
{
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
    pending.clear();
    used = 0;
}

// ---------------------------------------------------------------------------
// Graph residency: validate, orient, drop self-loops, merge duplicates, sort
// arcs by (dst, time, src), upload.  E^tau is a set of triples (Sec. 4).
// ---------------------------------------------------------------------------
Status build_graph(const tmotif_graph_desc *d, Graph *g)
{
    if (!d) return fail(TMOTIF_ERR_INVALID, "null graph descriptor");
    if (d->num_colors == 0) return fail(TMOTIF_ERR_INVALID, "num_colors must be >= 1");
    if (d->n > 0 && !d->color) return fail(TMOTIF_ERR_INVALID, "null color array");
    if (d->m > 0 && (!d->src || !d->dst || !d->time)) return fail(TMOTIF_ERR_INVALID, "null edge array");
    const u64 cap = d->undirected ? 2 * d->m : d->m;
    if (cap >= 0xFFFFFFFFull) return fail(TMOTIF_ERR_UNSUPPORTED, "more than 2^32-2 arcs");
    return build_graph_device(d, g);
}

void release_graph_arrays(Graph *g)
{
    if (!g) return;
    dev_free(g->d_src, g->stream);
    dev_free(g->d_dst, g->stream);
    dev_free(g->d_time, g->stream);
    dev_free(g->d_color, g->stream);
    dev_free(g->d_in_off, g->stream);
    g->d_src = g->d_dst = g->d_time = g->d_color = g->d_in_off = nullptr;
    dev_free(g->s_in, g->stream);
    dev_free(g->s_out, g->stream);
    g->s_in = g->s_out = nullptr;
    g->s_built = false;
    g->m_static = 0;
    g->sw.release();
    g->ws.release();
    cudaStreamSynchronize(g->stream);
    g->prof.destroy();
}

static void free_graph(Graph *g)
{
    if (!g) return;
    release_graph_arrays(g);
    delete static_cast<tmotif_graph *>(g);
}

Status parse_query(const Graph &g, const tmotif_query *q, QuerySpec *out)
{
    if (!q) return fail(TMOTIF_ERR_INVALID, "null query");
    if (q->k < 2 || q->k > TMOTIF_KMAX)
        return fail(TMOTIF_ERR_UNSUPPORTED, "k must be in [2, " + std::to_string(TMOTIF_KMAX) + "]");
    if (!q->multiset) return fail(TMOTIF_ERR_INVALID, "null multiset");
    if (q->repeats < 1) return fail(TMOTIF_ERR_INVALID, "repeats must be >= 1");
    if (q->start != TMOTIF_ANY && q->start >= g.n) return fail(TMOTIF_ERR_INVALID, "start vertex out of range");
    if (q->end != TMOTIF_ANY && q->end >= g.n) return fail(TMOTIF_ERR_INVALID, "end vertex out of range");
    out->k = q->k;
    out->multiset.assign(q->multiset, q->multiset + q->k);
    for (u32 c : out->multiset)
        if (c >= g.num_colors) return fail(TMOTIF_ERR_INVALID, "multiset colour out of range");
    out->start = q->start;
    out->end = q->end;
    out->t_min = q->t_min;
    out->t_max = q->t_max;
    out->seed = q->seed;
    out->repeats = q->repeats;
    out->flags = q->flags;
    out->times_exact.clear();
    if (q->timestamps) {
        for (u32 i = 0; i + 1 < q->k; i++) {
            const u32 t = q->timestamps[i];
            if (t == 0 || (i > 0 && t <= q->timestamps[i - 1]))
                return fail(TMOTIF_ERR_INVALID, "EC timestamps must be k-1 strictly increasing times >= 1");
            out->times_exact.push_back(t);
        }
    }
    const u64 full = 1ull << q->k;
    if (q->point_begin == 0 && q->point_end == 0) {
        out->p_begin = 0;
        out->p_end = full;
    } else {
        if (q->point_begin >= q->point_end || q->point_end > full)
            return fail(TMOTIF_ERR_INVALID, "bad point range");
        out->p_begin = q->point_begin;
        out->p_end = q->point_end;
    }
    return Status();
}

}  // namespace tmo

using namespace tmo;


extern "C" {

int tmotif_create_graph(const tmotif_graph_desc *desc, tmotif_graph_t *out)
{
    if (!out) return fail(TMOTIF_ERR_INVALID, "null output handle").code;
    *out = nullptr;
    tmotif_graph *g = nullptr;
    try {
        g = new tmotif_graph();
    } catch (const std::bad_alloc &) {
        return fail(TMOTIF_ERR_OOM, "host allocation failed").code;
    }
    Status s;
    try {
        if (desc) {
            g->stream = (cudaStream_t)desc->cuda_stream;
            g->ws.set_stream(g->stream);
        }
        s = build_graph(desc, g);
    } catch (const std::bad_alloc &) {
        s = fail(TMOTIF_ERR_OOM, "host allocation failed");
    }
    if (!s.ok()) {
        free_graph(g);
        return s.code;
    }
    *out = g;
    return TMOTIF_OK;
}

void tmotif_destroy_graph(tmotif_graph_t g) { free_graph(g); }

int tmotif_graph_get_info(tmotif_graph_t g, tmotif_graph_info *info)
{
    if (!g || !info) return fail(TMOTIF_ERR_INVALID, "null argument").code;
    info->n = g->n;
    info->m_input = g->m_input;
    info->m_arcs = g->m;
    info->self_loops = g->self_loops;
    info->duplicates = g->duplicates;
    info->max_time = g->max_time;
    info->device_bytes = g->resident_bytes + g->ws.bytes();
    return TMOTIF_OK;
}

}  // extern "C"

namespace {

// With TMOTIF_PREPROCESS_STATIC: the static sieve's kept vertices and the
// graph of the arcs among them (same vertex ids; Sec. 8.1 (ii) rebuilds the
// temporal graph on those vertices).  Otherwise the graph itself.
void delete_subgraph(Graph *x)
{
    release_graph_arrays(x);
    delete x;
}

struct Prepared {
    Graph *g = nullptr;
    std::unique_ptr<Graph, void (*)(Graph *)> sub{nullptr, delete_subgraph};
    double ms = 0;
};

// Add the statistics of work done on a preprocessed subgraph to its parent.
void merge_stats(Graph &g, const Prepared &p)
{
    if (!p.sub) return;
    const tmotif_stats &b = p.sub->prof.stats;
    tmotif_stats &a = g.prof.stats;
    a.launches += b.launches;
    a.layer_launches += b.layer_launches;
    a.layer_ms += b.layer_ms;
    a.prep_ms += b.prep_ms;
    a.coef_ms += b.coef_ms;
    a.other_ms += b.other_ms;
    a.layer_arc_lanes += b.layer_arc_lanes;
    a.layer_cp_lanes += b.layer_cp_lanes;
    a.layer_bytes += b.layer_bytes;
    a.layer_gf_muls += b.layer_gf_muls;
    a.layer_table_muls += b.layer_table_muls;
    a.layer_table_builds += b.layer_table_builds;
}

Status prepare(Graph &g, const QuerySpec &q, Prepared *p)
{
    p->g = &g;
    if (!(q.flags & TMOTIF_PREPROCESS_STATIC)) return Status();
    cudaEvent_t e0, e1;
    TM_CUDA(cudaEventCreate(&e0));
    TM_CUDA(cudaEventCreate(&e1));
    TM_CUDA(cudaEventRecord(e0, g.stream));
    g.sw.set_stream(g.stream);
    TM_TRY(g.sw.mask.reserve(std::max<u32>(g.n, 1)));
    TM_TRY(static_mask(g, q, nullptr, g.sw.mask.as<uint8_t>(), nullptr));
    p->sub.reset(new Graph());
    TM_TRY(make_subgraph(g, g.ws, g.stream, g.sw.mask.as<uint8_t>(), p->sub.get()));
    p->sub->prof.on = g.prof.on;  // its work is reported in g's statistics
    TM_CUDA(cudaEventRecord(e1, g.stream));
    TM_CUDA(cudaEventSynchronize(e1));
    float f = 0;
    cudaEventElapsedTime(&f, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->ms = f;
    p->g = p->sub.get();
    TM_TRY(g.prof.collect());  // the static sieve's events, recorded on g
    return Status();
}

}  // namespace

extern "C" {

int tmotif_decide(tmotif_graph_t g, const tmotif_query *q, tmotif_decision *out)
{
    if (!g || !out) return fail(TMOTIF_ERR_INVALID, "null argument").code;
    try {
        QuerySpec qs;
        Status s = parse_query(*g, q, &qs);
        if (!s.ok()) return s.code;
        Prepared pre;
        s = prepare(*g, qs, &pre);
        if (!s.ok()) return s.code;
        int found = 0;
        u64 sum = 0;
        double ms = 0;
        s = sieve_decide(*pre.g, qs, nullptr, &found, &sum, (u64 *)out->per_point, &ms);
        merge_stats(*g, pre);
        if (!s.ok()) return s.code;
        out->found = found;
        out->sieve_sum = sum;
        out->ms = ms + pre.ms;
        return TMOTIF_OK;
    } catch (const std::bad_alloc &) {
        return fail(TMOTIF_ERR_OOM, "host allocation failed").code;
    }
}

int tmotif_extract(tmotif_graph_t g, const tmotif_query *q, uint32_t *verts, uint32_t *times, int *found)
{
    if (!g || !verts || !times || !found) return fail(TMOTIF_ERR_INVALID, "null argument").code;
    try {
        QuerySpec qs;
        Status s = parse_query(*g, q, &qs);
        if (!s.ok()) return s.code;
        if (qs.p_begin != 0 || qs.p_end != (1ull << qs.k))
            return fail(TMOTIF_ERR_INVALID, "extraction needs the full point range").code;
        Prepared pre;
        s = prepare(*g, qs, &pre);
        if (!s.ok()) return s.code;
        Graph &G = *pre.g;
        if (qs.flags & TMOTIF_EXTRACT_OPTIMUM) {
            u32 t_opt = 0;
            int any = 0;
            s = optimum_time(G, qs, &t_opt, &any);
            if (!s.ok()) return s.code;
            if (!any) {
                *found = 0;
                merge_stats(*g, pre);
                return TMOTIF_OK;
            }
            qs.t_max = t_opt;
        }
        if (qs.flags & TMOTIF_EXTRACT_HALVING) {
            u32 probes = 0;
            s = extract_path(G, qs, verts, times, found, &probes);
        } else {
            s = extract_localized(G, qs, verts, times, found);
        }
        merge_stats(*g, pre);
        return s.code;
    } catch (const std::bad_alloc &) {
        return fail(TMOTIF_ERR_OOM, "host allocation failed").code;
    }
}

int tmotif_optimum_time(tmotif_graph_t g, const tmotif_query *q, uint32_t *t_opt, int *found)
{
    if (!g || !t_opt || !found) return fail(TMOTIF_ERR_INVALID, "null argument").code;
    try {
        QuerySpec qs;
        Status s = parse_query(*g, q, &qs);
        if (!s.ok()) return s.code;
        if (qs.p_begin != 0 || qs.p_end != (1ull << qs.k))
            return fail(TMOTIF_ERR_INVALID, "the optimum time needs the full point range").code;
        Prepared pre;
        s = prepare(*g, qs, &pre);
        if (!s.ok()) return s.code;
        s = optimum_time(*pre.g, qs, t_opt, found);
        merge_stats(*g, pre);
        return s.code;
    } catch (const std::bad_alloc &) {
        return fail(TMOTIF_ERR_OOM, "host allocation failed").code;
    }
}

int tmotif_localize(tmotif_graph_t g, const tmotif_query *q, uint64_t *per_vertex, tmotif_decision *out)
{
    if (!g || !per_vertex || !out) return fail(TMOTIF_ERR_INVALID, "null argument").code;
    try {
        QuerySpec qs;
        Status s = parse_query(*g, q, &qs);
        if (!s.ok()) return s.code;
        if (qs.p_begin != 0 || qs.p_end != (1ull << qs.k))
            return fail(TMOTIF_ERR_INVALID, "localisation needs the full point range").code;
        Prepared pre;
        s = prepare(*g, qs, &pre);
        if (!s.ok()) return s.code;
        int found = 0;
        u64 sum = 0;
        double ms = 0;
        s = sieve_localize(*pre.g, qs, (u64 *)per_vertex, &found, &sum, &ms);
        merge_stats(*g, pre);
        if (!s.ok()) return s.code;
        out->found = found;
        out->sieve_sum = sum;
        out->ms = ms + pre.ms;
        return TMOTIF_OK;
    } catch (const std::bad_alloc &) {
        return fail(TMOTIF_ERR_OOM, "host allocation failed").code;
    }
}

int tmotif_static_sieve(tmotif_graph_t g, const tmotif_query *q, uint64_t *per_vertex, uint32_t *kept)
{
    if (!g) return fail(TMOTIF_ERR_INVALID, "null graph").code;
    try {
        QuerySpec qs;
        Status s = parse_query(*g, q, &qs);
        if (!s.ok()) return s.code;
        g->sw.set_stream(g->stream);
        s = g->sw.qv.reserve(std::max<u32>(g->n, 1) * 8ull);
        if (!s.ok()) return s.code;
        s = static_sieve(*g, qs, nullptr, g->sw.qv.as<u64>(), nullptr);
        if (!s.ok()) return s.code;
        std::vector<u64> h(g->n);
        if (g->n) {
            cudaError_t e = cudaMemcpyAsync(h.data(), g->sw.qv.p, (u64)g->n * 8, cudaMemcpyDeviceToHost, g->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
            if (e != cudaSuccess) return cuda_fail(e, "static sieve readback").code;
        }
        if (per_vertex && g->n) std::memcpy(per_vertex, h.data(), (u64)g->n * 8);
        if (kept) {
            u32 c = 0;
            for (u64 v : h) c += v != 0;
            *kept = c;
        }
        return g->prof.collect().code;
    } catch (const std::bad_alloc &) {
        return fail(TMOTIF_ERR_OOM, "host allocation failed").code;
    }
}

int tmotif_set_profiling(tmotif_graph_t g, int on)
{
    if (!g) return fail(TMOTIF_ERR_INVALID, "null graph").code;
    g->prof.on = on != 0;
    std::memset(&g->prof.stats, 0, sizeof(g->prof.stats));
    g->prof.pending.clear();
    g->prof.used = 0;
    return TMOTIF_OK;
}


uint32_t tmotif_checked_build(void)
{
#ifdef TMOTIF_CHECKED
    return 1;
#else
    return 0;
#endif
}

int tmotif_set_layer_shape(tmotif_graph_t g, uint32_t L, uint32_t chunk, uint32_t variant)
{
    if (!g) return fail(TMOTIF_ERR_INVALID, "null graph").code;
    if (!layer_shape_valid(L, chunk, variant)) return fail(TMOTIF_ERR_INVALID, "bad layer shape").code;
    std::lock_guard<std::mutex> lock(layer_tune_mutex());
    g->layer_tune[L] = {chunk, variant};
    return TMOTIF_OK;
}

int tmotif_get_layer_shape(tmotif_graph_t g, uint32_t L, uint32_t *chunk, uint32_t *variant)
{
    if (!g || !chunk || !variant) return fail(TMOTIF_ERR_INVALID, "null argument").code;
    std::lock_guard<std::mutex> lock(layer_tune_mutex());
    auto it = g->layer_tune.find(L);
    if (it == g->layer_tune.end()) return fail(TMOTIF_ERR_NOT_FOUND, "no layer shape for this lane width").code;
    *chunk = it->second.first;
    *variant = it->second.second;
    return TMOTIF_OK;
}

int tmotif_get_stats(tmotif_graph_t g, tmotif_stats *out)
{
    if (!g || !out) return fail(TMOTIF_ERR_INVALID, "null argument").code;
    *out = g->prof.stats;
    return TMOTIF_OK;
}

int tmotif_gf_mul_batch(const uint64_t *a, const uint64_t *b, uint64_t *out, uint64_t n)
{
    if (n && (!a || !b || !out)) return fail(TMOTIF_ERR_INVALID, "null argument").code;
    return gf_mul_batch((const u64 *)a, (const u64 *)b, (u64 *)out, n).code;
}

int tmotif_debug_stage_timeout(int on) { return debug_stage_timeout(on != 0).code; }

int tmotif_memory_stats(uint64_t *used, uint64_t *used_high, uint64_t *reserved, int reset)
{
    return memory_stats((u64 *)used, (u64 *)used_high, (u64 *)reserved, reset != 0).code;
}

int tmotif_tuner_export(char *buf, size_t cap, size_t *len)
{
    if (!len || (cap && !buf)) return fail(TMOTIF_ERR_INVALID, "null argument").code;
    try {
        const std::string t = tuner_export();
        *len = t.size();
        if (cap) {
            const size_t n = std::min(cap - 1, t.size());
            std::memcpy(buf, t.data(), n);
            buf[n] = 0;
        }
        return TMOTIF_OK;
    } catch (const std::bad_alloc &) {
        return fail(TMOTIF_ERR_OOM, "host allocation failed").code;
    }
}

int tmotif_tuner_import(const char *text)
{
    if (!text) return fail(TMOTIF_ERR_INVALID, "null text").code;
    try {
        return tuner_import(text).code;
    } catch (const std::bad_alloc &) {
        return fail(TMOTIF_ERR_OOM, "host allocation failed").code;
    }
}

int tmotif_gf_probe(int method, uint32_t iters, double *ms, uint64_t *products)
{
    if (!ms || !products || method < 0 || method > 2 || iters == 0)
        return fail(TMOTIF_ERR_INVALID, "bad probe arguments").code;
    return gf_probe(method, iters, ms, (u64 *)products).code;
}

const char *tmotif_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
