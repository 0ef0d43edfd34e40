// extract.cu -- extraction of a matching temporal path (Sec. 6.9).
//
// Step (i), self-reducibility with halving: the candidate set R holds the
// vertices whose colour is in M, in ascending id.  shrink(block) removes the
// block when the query is still YES without it (a decision on the graph with
// those vertices masked, x_u = 0), otherwise halves a block of more than one
// candidate and tries both halves in order.  A block that holds every
// remaining candidate is not probed (removing it leaves no path).  Probe i
// uses seed mix64(seed ^ i * TM_PROBE).  Step (ii): a temporal DFS on the
// survivors, start vertices in ascending id, arcs in (time, dst) order,
// returns the first path whose colours are M.
//
// The halving runs as a state machine over an explicit stack of blocks
// (popped in the order the recursion would visit them), so a caller can run
// the probes one at a time -- synchronously here, or interleaved with other
// work in the request server.
#include <algorithm>
#include <map>
#include <numeric>
#include <mutex>
#include <vector>

#include "gf64.cuh"
#include "internal.h"

namespace tmo {

Status ensure_host_colors(Graph &g)
{
    static std::mutex mu;  // the server's lanes and submitting threads share graphs
    std::lock_guard<std::mutex> lock(mu);
    if (g.h_color) return Status();
    auto c = std::make_shared<std::vector<u32>>(g.n);
    if (g.n) {
        TM_CUDA(cudaMemcpyAsync(c->data(), g.d_color, (u64)g.n * 4, cudaMemcpyDeviceToHost, g.stream));
        TM_CUDA(cudaStreamSynchronize(g.stream));
    }
    g.h_color = std::move(c);
    return Status();
}

void ExtractState::init(const Graph &g, const QuerySpec &q)
{
    query = q;
    std::vector<uint8_t> in_m(g.num_colors, 0);
    for (u32 c : q.multiset) in_m[c] = 1;
    alive.assign(g.n, 0);
    R.clear();
    for (u32 u = 0; u < g.n; u++)
        if (in_m[(*g.h_color)[u]]) {
            alive[u] = 1;
            R.push_back(u);
        }
    n_alive = R.size();
    alive_at_build = n_alive;
    sub.reset();
    stack.clear();
    stack.push_back({0, (u64)R.size()});
    probes = 0;
    stage = FIRST;
    cur_lo = cur_hi = 0;
    cur_cnt = 0;
}

bool ExtractState::next_probe(QuerySpec *pq)
{
    if (stage == FIRST) {
        *pq = query;
        return true;
    }
    if (stage == NOT_FOUND || stage == SHRUNK) return false;
    while (!stack.empty()) {
        const Block b = stack.back();
        stack.pop_back();
        u64 cnt = 0;
        for (u64 i = b.lo; i < b.hi; i++) cnt += alive[R[i]];
        if (cnt == 0) continue;
        if (cnt < n_alive) {
            for (u64 i = b.lo; i < b.hi; i++) alive[R[i]] = 0;
            probes++;
            cur_lo = b.lo;
            cur_hi = b.hi;
            cur_cnt = cnt;
            *pq = query;
            pq->seed = mix64(query.seed ^ ((u64)probes * TM_PROBE));
            pq->p_begin = 0;
            pq->p_end = 1ull << query.k;
            stage = PROBING;
            return true;
        }
        push_halves(b.lo, b.hi);
    }
    stage = SHRUNK;
    return false;
}

void ExtractState::push_halves(u64 lo, u64 hi)
{
    if (hi - lo <= 1) return;
    const u64 mid = lo + (hi - lo) / 2;
    stack.push_back({mid, hi});  // visited second
    stack.push_back({lo, mid});  // visited first
}

void ExtractState::result(bool yes)
{
    if (stage == FIRST) {
        stage = yes ? SEARCHING : NOT_FOUND;
        return;
    }
    if (yes) {
        n_alive -= cur_cnt;
    } else {
        // a block is probed before its sub-blocks, so all of it was alive
        for (u64 i = cur_lo; i < cur_hi; i++) alive[R[i]] = 1;
        push_halves(cur_lo, cur_hi);
    }
    stage = SEARCHING;
}

Status ExtractState::maybe_compact(Graph &root, Workspace &w, cudaStream_t st)
{
    if (2 * n_alive > alive_at_build) return Status();
    // the survivors so far, with the block under probe still in: a probe
    // that answers NO puts it back
    std::vector<uint8_t> keep = alive;
    if (stage == PROBING)
        for (u64 i = cur_lo; i < cur_hi; i++) keep[R[i]] = 1;
    TM_TRY(w.alive.reserve(std::max<size_t>(keep.size(), 1)));
    TM_CUDA(cudaMemcpyAsync(w.alive.p, keep.data(), keep.size(), cudaMemcpyHostToDevice, st));
    std::unique_ptr<Graph, void (*)(Graph *)> next(new Graph(), [](Graph *g) {
        release_graph_arrays(g);
        delete g;
    });
    TM_TRY(make_subgraph(*current(root), w, st, w.alive.as<uint8_t>(), next.get()));
    sub = std::move(next);
    alive_at_build = n_alive;
    return Status();
}

namespace {

struct Dfs {
    const QuerySpec *q;
    const std::vector<u32> *color;
    std::map<u32, std::vector<std::pair<u32, u32>>> out;  // src -> [(time, dst)]
    std::map<u32, u32> need;
    std::vector<u32> walk, wt;
    std::map<u32, bool> onpath;
    bool found = false;

    bool rec(u32 depth, u32 last_t)
    {
        if (depth == q->k) {
            if (q->end != TMOTIF_ANY && walk[q->k - 1] != q->end) return false;
            found = true;
            return true;
        }
        auto it = out.find(walk[depth - 1]);
        if (it == out.end()) return false;
        for (const auto &tv : it->second) {
            const u32 t = tv.first, v = tv.second;
            if (t <= last_t || onpath[v]) continue;
            const u32 c = (*color)[v];
            auto nd = need.find(c);
            if (nd == need.end() || nd->second == 0) continue;
            nd->second--;
            onpath[v] = true;
            walk[depth] = v;
            wt[depth - 1] = t;
            bool stop = rec(depth + 1, t);
            nd->second++;
            onpath[v] = false;
            if (stop) return true;
        }
        return false;
    }
};

}  // namespace

// (ii) temporal DFS on the survivors, whose arcs are gathered on the device.
Status extract_finish(Graph &g, Workspace &w, cudaStream_t st, Profiler &prof, const ExtractState &ex, u32 *verts,
                      u32 *times, int *found)
{
    const QuerySpec &q = ex.query;
    *found = 0;
    TM_TRY(w.alive.reserve(std::max<u32>(g.n, 1)));
    TM_CUDA(cudaMemcpyAsync(w.alive.p, ex.alive.data(), g.n, cudaMemcpyHostToDevice, st));
    std::vector<u32> as, ad, at;
    TM_TRY(gather_arcs(g, w, st, prof, w.alive.as<uint8_t>(), q.filter(), &as, &ad, &at));
    Dfs D;
    D.q = &q;
    D.color = g.h_color.get();
    std::vector<size_t> idx(as.size());
    std::iota(idx.begin(), idx.end(), 0);
    std::sort(idx.begin(), idx.end(), [&](size_t x, size_t y) {
        if (at[x] != at[y]) return at[x] < at[y];
        if (as[x] != as[y]) return as[x] < as[y];
        return ad[x] < ad[y];
    });
    for (size_t i : idx) D.out[as[i]].push_back({at[i], ad[i]});
    for (u32 c : q.multiset) D.need[c]++;
    D.walk.assign(q.k, 0);
    D.wt.assign(q.k, 0);
    for (u32 u = 0; u < g.n && !D.found; u++) {
        if (!ex.alive[u]) continue;
        if (q.start != TMOTIF_ANY && u != q.start) continue;
        auto nd = D.need.find((*g.h_color)[u]);
        if (nd == D.need.end() || nd->second == 0) continue;
        nd->second--;
        D.onpath[u] = true;
        D.walk[0] = u;
        D.rec(1, 0);
        nd->second++;
        D.onpath[u] = false;
    }
    if (D.found) {
        for (u32 r = 0; r < q.k; r++) verts[r] = D.walk[r];
        for (u32 r = 0; r + 1 < q.k; r++) times[r] = D.wt[r];
        *found = 1;
    }
    return Status();
}

Status extract_path(Graph &g, const QuerySpec &q, u32 *verts, u32 *times, int *found, u32 *probes)
{
    *found = 0;
    *probes = 0;
    ExtractState ex;
    TM_TRY(ensure_host_colors(g));
    ex.init(g, q);
    TM_TRY(g.ws.alive.reserve(std::max<u32>(g.n, 1)));
    QuerySpec pq;
    while (ex.next_probe(&pq)) {
        const uint8_t *mask = nullptr;
        Graph *cur = &g;
        if (ex.stage == ExtractState::PROBING) {
            TM_TRY(ex.maybe_compact(g, g.ws, g.stream));
            cur = ex.current(g);
            TM_TRY(cur->ws.alive.reserve(std::max<u32>(g.n, 1)));
            TM_CUDA(cudaMemcpyAsync(cur->ws.alive.p, ex.alive.data(), g.n, cudaMemcpyHostToDevice, cur->stream));
            mask = cur->ws.alive.as<uint8_t>();
        }
        int yes = 0;
        u64 sum = 0;
        double ms = 0;
        TM_TRY(sieve_decide(*cur, pq, mask, &yes, &sum, nullptr, &ms));
        ex.result(yes != 0);
        if (ex.stage == ExtractState::NOT_FOUND) return Status();
    }
    *probes = ex.probes;
    Graph *cur = ex.current(g);
    return extract_finish(*cur, cur->ws, cur->stream, cur->prof, ex, verts, times, found);
}

// ---------------------------------------------------------------------------
// Extraction by localisation (Sec. 6.9, second approach, localised to arcs).
// Level 1: the arc-localised sieve of the query; its first nonzero arc
// (a1 -> b1, t1) in (dst, time, src) order ends a matching path.  Level j:
// a path on the remaining colours ending at a_{j-1}, every time below
// t_{j-1}, the vertices chosen after a_{j-1} masked; its first nonzero arc
// into a_{j-1} extends the path backwards.  Level j evaluates with seed
// mix64(seed ^ j * TM_PROBE); with repeats > 1 an arc counts when any repeat
// is nonzero, and the first such arc is taken.
// ---------------------------------------------------------------------------
void LocalizedExtract::init(const Graph &g, const QuerySpec &q)
{
    query = q;
    color = g.h_color;
    ms = q.multiset;
    alive.assign(g.n, 1);
    verts.assign(q.k, 0);
    times.assign(q.k, 0);
    kk = q.k;
    level = 1;
    rep = 0;
    cur_end = q.end;
    cur_tmax = q.t_max;
    best = NONE;
    done = false;
    found = false;
}

bool LocalizedExtract::next(QuerySpec *sub, u32 *repeat, const std::vector<uint8_t> **mask)
{
    if (done) return false;
    *sub = query;
    sub->k = kk;
    sub->multiset.assign(ms.begin(), ms.begin() + kk);
    sub->end = cur_end;
    sub->t_max = cur_tmax;
    sub->seed = mix64(query.seed ^ ((u64)level * TM_PROBE));
    sub->repeats = 1;
    sub->p_begin = 0;
    sub->p_end = 1ull << kk;
    *repeat = rep;
    *mask = level > 1 ? &alive : nullptr;
    return true;
}

void LocalizedExtract::result(u32 idx, u32 a, u32 b, u32 t)
{
    if (idx != NONE && idx < best) {
        best = idx;
        ba = a;
        bb = b;
        bt = t;
    }
    if (++rep < query.repeats) return;  // more repeats of this level
    rep = 0;
    if (best == NONE) {  // no path (or a false negative)
        done = true;
        return;
    }
    if (level == 1) verts[query.k - 1] = bb;
    verts[kk - 2] = ba;
    times[kk - 2] = bt;
    // bb's colour leaves the multiset and bb leaves the graph
    const u32 cb = (*color)[bb];
    for (u32 r = 0; r < kk; r++)
        if (ms[r] == cb) {
            ms[r] = ms[kk - 1];
            break;
        }
    kk--;
    alive[bb] = 0;
    best = NONE;
    if (kk < 2) {
        found = true;
        done = true;
        return;
    }
    if (bt <= 1) {  // nothing can come before time 1
        done = true;
        return;
    }
    cur_end = ba;
    cur_tmax = bt - 1;
    level++;
}

Status extract_localized(Graph &g, const QuerySpec &q, u32 *verts, u32 *times, int *found)
{
    *found = 0;
    LocalizedExtract ex;
    TM_TRY(ensure_host_colors(g));
    ex.init(g, q);
    QuerySpec sub;
    u32 rep = 0;
    const std::vector<uint8_t> *mask = nullptr;
    while (ex.next(&sub, &rep, &mask)) {
        const uint8_t *d_mask = nullptr;
        if (mask) {
            TM_TRY(g.ws.alive.reserve(std::max<u32>(g.n, 1)));
            TM_CUDA(cudaMemcpyAsync(g.ws.alive.p, mask->data(), g.n, cudaMemcpyHostToDevice, g.stream));
            d_mask = g.ws.alive.as<uint8_t>();
        }
        u32 best = NONE, a = 0, b = 0, t = 0;
        TM_TRY(sieve_first_arc(g, sub, rep, d_mask, &best, &a, &b, &t));
        ex.result(best, a, b, t);
    }
    if (ex.found) {
        for (u32 r = 0; r < q.k; r++) verts[r] = ex.verts[r];
        for (u32 r = 0; r + 1 < q.k; r++) times[r] = ex.times[r];
        *found = 1;
    }
    return Status();
}

Status optimum_time(Graph &g, const QuerySpec &q, u32 *t_opt, int *found)
{
    *found = 0;
    *t_opt = 0;
    u32 lo = q.t_min > 1 ? q.t_min : 1, hi = q.t_max ? q.t_max : g.max_time;
    if (hi < lo || g.m == 0) return Status();
    QuerySpec p = q;
    p.t_max = hi;
    int yes = 0;
    u64 sum = 0;
    double ms = 0;
    TM_TRY(sieve_decide(g, p, nullptr, &yes, &sum, nullptr, &ms));
    if (!yes) return Status();
    while (lo < hi) {
        const u32 mid = lo + (hi - lo) / 2;
        p.t_max = mid;
        TM_TRY(sieve_decide(g, p, nullptr, &yes, &sum, nullptr, &ms));
        if (yes) hi = mid;
        else lo = mid + 1;
    }
    *found = 1;
    *t_opt = lo;
    return Status();
}

}  // namespace tmo
