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
#include <algorithm>
#include <functional>
#include <map>
#include <numeric>
#include <vector>

#include "gf64.cuh"
#include "internal.h"

namespace tmo {

namespace {

struct Dfs {
    const QuerySpec *q;
    const std::vector<u32> *color;
    // out-arcs per vertex in (time, dst) order
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

Status extract_path(Graph &g, const QuerySpec &q, u32 *verts, u32 *times, int *found, u32 *probes)
{
    *found = 0;
    *probes = 0;
    const u32 n = g.n;
    std::vector<uint8_t> in_m(g.num_colors, 0);
    for (u32 c : q.multiset) in_m[c] = 1;
    std::vector<uint8_t> alive(n, 0);
    std::vector<u32> R;
    for (u32 u = 0; u < n; u++)
        if (in_m[g.h_color[u]]) {
            alive[u] = 1;
            R.push_back(u);
        }

    int yes = 0;
    u64 sum = 0;
    double ms = 0;
    TM_TRY(sieve_decide(g, q, nullptr, &yes, &sum, nullptr, &ms));
    if (!yes) return Status();

    TM_TRY(g.ws.alive.reserve(std::max<u32>(n, 1)));
    u64 n_alive = R.size();
    u32 probe = 0;
    Status err;
    std::function<void(u64, u64)> shrink = [&](u64 lo, u64 hi) {
        if (!err.ok()) return;
        u64 cnt = 0;
        for (u64 i = lo; i < hi; i++) cnt += alive[R[i]];
        if (cnt == 0) return;
        if (cnt < n_alive) {
            for (u64 i = lo; i < hi; i++) alive[R[i]] = 0;
            probe++;
            cudaError_t e = cudaMemcpyAsync(g.ws.alive.p, alive.data(), n, cudaMemcpyHostToDevice, g.stream);
            if (e != cudaSuccess) { err = cuda_fail(e, "probe mask upload"); return; }
            QuerySpec pq = q;
            pq.seed = mix64(q.seed ^ ((u64)probe * TM_PROBE));
            pq.p_begin = 0;
            pq.p_end = 1ull << q.k;
            int py = 0;
            Status s = sieve_decide(g, pq, g.ws.alive.as<uint8_t>(), &py, &sum, nullptr, &ms);
            if (!s.ok()) { err = s; return; }
            if (py) {
                n_alive -= cnt;
                return;
            }
            // a block is probed before its sub-blocks, so all of it was alive
            for (u64 i = lo; i < hi; i++) alive[R[i]] = 1;
        }
        if (hi - lo == 1) return;
        const u64 mid = lo + (hi - lo) / 2;
        shrink(lo, mid);
        shrink(mid, hi);
    };
    shrink(0, R.size());
    TM_TRY(err);
    *probes = probe;

    // (ii) temporal DFS on the survivors
    TM_CUDA(cudaMemcpyAsync(g.ws.alive.p, alive.data(), n, cudaMemcpyHostToDevice, g.stream));
    std::vector<u32> as, ad, at;
    TM_TRY(gather_arcs(g, g.ws.alive.as<uint8_t>(), q.t_min, q.t_max, &as, &ad, &at));
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
    for (u32 u = 0; u < n && !D.found; u++) {
        if (!alive[u]) continue;
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

}  // namespace tmo
