// extract.cu -- extraction of a matching temporal path (Sec. 5.9).
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
#include <vector>

#include "gf64.cuh"
#include "internal.h"

namespace tmo {

void ExtractState::init(const Graph &g, const QuerySpec &q)
{
    query = q;
    std::vector<uint8_t> in_m(g.num_colors, 0);
    for (u32 c : q.multiset) in_m[c] = 1;
    alive.assign(g.n, 0);
    R.clear();
    for (u32 u = 0; u < g.n; u++)
        if (in_m[g.h_color[u]]) {
            alive[u] = 1;
            R.push_back(u);
        }
    n_alive = R.size();
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
    TM_TRY(gather_arcs(g, w, st, prof, w.alive.as<uint8_t>(), q.t_min, q.t_max, &as, &ad, &at));
    Dfs D;
    D.q = &q;
    D.color = &g.h_color;
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
        auto nd = D.need.find(g.h_color[u]);
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
    ex.init(g, q);
    TM_TRY(g.ws.alive.reserve(std::max<u32>(g.n, 1)));
    QuerySpec pq;
    while (ex.next_probe(&pq)) {
        const uint8_t *mask = nullptr;
        if (ex.stage == ExtractState::PROBING) {
            TM_CUDA(cudaMemcpyAsync(g.ws.alive.p, ex.alive.data(), g.n, cudaMemcpyHostToDevice, g.stream));
            mask = g.ws.alive.as<uint8_t>();
        }
        int yes = 0;
        u64 sum = 0;
        double ms = 0;
        TM_TRY(sieve_decide(g, pq, mask, &yes, &sum, nullptr, &ms));
        ex.result(yes != 0);
        if (ex.stage == ExtractState::NOT_FOUND) return Status();
    }
    *probes = ex.probes;
    return extract_finish(g, g.ws, g.stream, g.prof, ex, verts, times, found);
}

}  // namespace tmo
