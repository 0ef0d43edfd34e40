// pack.cu -- packed many-graph batches.
//
// A batch of many small graphs, each with its own query, runs as one packed
// problem:
// - the graphs' canonical arcs are copied into one arc array with vertex ids
//   offset per graph (graph i owns packed vertices [vbase_i, vbase_i + n_i)),
//   so every in-segment, predecessor arc and checkpoint stays inside its
//   graph and the per-query filter, segment, predecessor and checkpoint
//   kernels of a single query run unchanged, once, for the whole batch;
// - the coefficients x_u^A use each graph's own vertex ids, keys and slots;
// - y uses each query's key and the graph's own vertex ids;
// - one layer launch per walk length serves every query: a segment's query
//   decides whether the layer is inside its walk, its last layer, or past it.
// So every value equals the one tmotif_decide computes for that graph and
// query alone.  Lane batches: round r evaluates points [64 r, 64 r + 64) of
// every query that has them; lanes past a query's 2^k points are ignored.
#include <algorithm>
#include <cstring>

#include "gf64.cuh"
#include "internal.h"
#include "layer.cuh"
#include "scan.cuh"

namespace tmo {

// per-query kernels reused from sieve.cu
__global__ void k_active_list(u32 n, const u32 *act, u32 *list);
__global__ void k_compact(u64 m, const u32 *src, const u32 *dst, const u32 *time, const u32 *off, u32 *f_src,
                          u32 *f_dst, u32 *f_time);
__global__ void k_segments(u64 mf, const u32 *f_dst, u32 *seg_lo, u32 *seg_hi, u32 n);
__global__ void k_pos(u64 mf, const u32 *f_src, const u32 *f_time, const u32 *seg_lo, const u32 *seg_hi, u32 *pos,
                      u32 *mark, u32 n);
__global__ void k_checkpoints(u64 mf, const u32 *pos, const u32 *ck, u32 *cp_in, u32 *cp_out, const u32 *f_src,
                              const u32 *f_dst, uint4 *rec, const u32 *seg_hi, u32 *max_seg);

namespace {

const u32 PL = 64;                 // lanes per round
const u32 PCHUNK = 128;            // arcs per team chunk
const u64 PACK_ARCS = 120000000;   // arcs per pack (larger batches run as several packs)

// Where graph g's arrays sit and how they map into the packed numbering.
struct PackGraph {
    const u32 *src, *dst, *time, *color;
    u64 abase, m;
    u32 vbase, n;
};

// Per query: filter, slots, coefficient keys and table offsets.
struct PackQuery {
    ArcFilter filter;
    QueryKeys keys;
    u32 slot_off, wtab_off, npts, k;
};

unsigned blocks_of(u64 items, int threads) { return (unsigned)std::max<u64>(1, (items + threads - 1) / threads); }

// One block per graph: its arcs and vertices into the packed arrays.
__global__ void k_pack_gather(const PackGraph *gs, u32 *P_src, u32 *P_dst, u32 *P_time, u32 *P_color, u32 *jv)
{
    const PackGraph G = gs[blockIdx.x];
    for (u64 e = threadIdx.x; e < G.m; e += blockDim.x) {
        P_src[G.abase + e] = G.src[e] + G.vbase;
        P_dst[G.abase + e] = G.dst[e] + G.vbase;
        P_time[G.abase + e] = G.time[e];
    }
    for (u32 u = threadIdx.x; u < G.n; u += blockDim.x) {
        P_color[G.vbase + u] = G.color[u];
        jv[G.vbase + u] = blockIdx.x;
    }
}

// vflag[u] = u's query has points in this round and u's colour is in its
// multiset; act[] the same as u32 flags (N+1 entries) for the active list.
__global__ void k_pack_vflag(u32 N, const u32 *color, const u32 *jv, const PackQuery *qs, const u32 *slot_count,
                             u32 p0, uint8_t *vflag, u32 *act)
{
    const u64 u = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (u > N) return;
    if (u == N) { act[N] = 0; return; }
    const PackQuery &Q = qs[jv[u]];
    const bool f = p0 < Q.npts && slot_count[Q.slot_off + color[u]] > 0;
    vflag[u] = f ? 1 : 0;
    act[u] = f ? 1u : 0u;
}

// Arcs between flagged vertices that pass their query's window (and EC times).
__global__ void k_pack_keep(u64 M, const u32 *src, const u32 *dst, const u32 *time, const uint8_t *vflag,
                            const u32 *jv, const PackQuery *qs, u32 *keep)
{
    const u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (e > M) return;
    if (e == M) { keep[M] = 0; return; }
    const u32 d = dst[e];
    bool k = vflag[d] && vflag[src[e]];  // destinations are sorted: the source is read only when needed
    if (k) {
        const ArcFilter &f = qs[jv[d]].filter;
        const u32 t = time[e];
        k = t >= f.t_min && (f.t_max == 0 || t <= f.t_max);
        if (k && f.n_times) {
            bool in = false;
            for (u32 i = 0; i < f.n_times; i++) in |= (f.times[i] == t);
            k = in;
        }
    }
    keep[e] = k ? 1u : 0u;
}

// W_d^A of every query with points in this round: wtab[wtab_off + d * PL + lane].
__global__ void k_pack_wtab(u32 nq, const PackQuery *qs, u32 p0, u64 *wtab)
{
    const u32 qi = blockIdx.x;
    const PackQuery &Q = qs[qi];
    if (p0 >= Q.npts) return;
    for (u32 i = threadIdx.x; i < Q.k * PL; i += blockDim.x) {
        const u32 d = i / PL, lane = i % PL;
        const u64 point = p0 + lane;
        u64 s = 0;
        for (u32 j = 0; j < Q.k; j++)
            if ((point >> j) & 1u) s ^= coef_w(Q.keys, d, j);
        wtab[Q.wtab_off + i] = s;
    }
}

// x_u^A for the active vertices, one warp per vertex, with the vertex's
// query (keys, slots, W table) and its graph's own vertex id.
__global__ void __launch_bounds__(256) k_pack_coef(u32 n_act, const u32 *list, const u32 *color, const u32 *jv,
                                                   const PackQuery *qs, const PackGraph *gs,
                                                   const u32 *slot_begin, const u32 *slot_count, const u64 *wtab,
                                                   u64 *x)
{
    __shared__ __align__(2048) u64 tabs[8][256];  // tables on 2 KB boundaries
    u64 *tab = tabs[threadIdx.x >> 5];
    const int tt = threadIdx.x & 31;
    const u64 v = (u64)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (v >= n_act) return;  // whole warp leaves together
    const u32 u = list[v], qi = jv[u];
    const PackQuery &Q = qs[qi];
    const u32 local = u - gs[qi].vbase, c = color[u];
    const u32 d0 = slot_begin[Q.slot_off + c], d1 = d0 + slot_count[Q.slot_off + c];
    u64 s0 = 0, s1 = 0;
    for (u32 d = d0; d < d1; d++) {
        __syncwarp();
        gf_table_build(tab, coef_v(Q.keys, local, d), tt, 32);
        __syncwarp();
        s0 ^= gf_table_mul(tab, wtab[Q.wtab_off + d * PL + tt]);
        s1 ^= gf_table_mul(tab, wtab[Q.wtab_off + d * PL + tt + 32]);
    }
    x[(u64)u * PL + tt] = s0;
    x[(u64)u * PL + tt + 32] = s1;
}

__global__ void __launch_bounds__(256) k_pack_layer(LayerParams p)
{
    extern __shared__ __align__(16) u64 smem[];
    const u32 sa = (u32)__cvta_generic_to_shared(smem);
    u64 *tab = smem + (((2048u - (sa & 2047u)) & 2047u) >> 3) + (size_t)(threadIdx.x / 32) * 256;
    // resident warps take chunks in order from the counter (p.queue, zeroed
    // before the launch): graphs of uneven size leave no tail of idle SMs
    for (;;) {
        unsigned long long t = 0;
        if ((threadIdx.x & 31) == 0) t = atomicAdd(p.queue, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= p.n_chunks) return;
        layer_team<32, true, 2, true>(p, t, tab);
    }
}

struct PackBuffers {
    DevBuf graphs, queries, jobs, slot_begin, slot_count;
    DevBuf P_src, P_dst, P_time, P_color, jv;
    DevBuf vflag, act, act_list, keep, f_src, f_dst, f_time, seg_lo, seg_hi, pos, mark, cp_in, cp_out;
    DevBuf g_src, g_dst, g_time;  // the other set of kept arcs (rounds alternate)
    DevBuf wtab, x, C0, C1, out, block_sums, counters, queue;
    void set_stream(cudaStream_t s)
    {
        DevBuf *all[] = {&graphs, &queries, &jobs, &slot_begin, &slot_count, &P_src, &P_dst, &P_time, &P_color,
                         &jv, &vflag, &act, &act_list, &keep, &f_src, &f_dst, &f_time, &seg_lo, &seg_hi, &pos,
                         &mark, &cp_in, &cp_out, &g_src, &g_dst, &g_time, &wtab, &x, &C0, &C1, &out, &block_sums,
                         &counters, &queue};
        for (DevBuf *b : all) b->stream = s;
    }
    void release()
    {
        DevBuf *all[] = {&graphs, &queries, &jobs, &slot_begin, &slot_count, &P_src, &P_dst, &P_time, &P_color,
                         &jv, &vflag, &act, &act_list, &keep, &f_src, &f_dst, &f_time, &seg_lo, &seg_hi, &pos,
                         &mark, &cp_in, &cp_out, &g_src, &g_dst, &g_time, &wtab, &x, &C0, &C1, &out, &block_sums,
                         &counters, &queue};
        for (DevBuf *b : all) b->release();
    }
};

// One pack: queries [first, last) of the batch.
Status run_pack(Graph *const *graphs, const QuerySpec *specs, size_t first, size_t last, cudaStream_t st,
                PackBuffers &B, void *pinned, std::vector<std::vector<u64>> *vals, u64 *launches)
{
    const size_t nq = last - first;
    std::vector<PackGraph> hg(nq);
    std::vector<PackQuery> hq(nq);
    std::vector<PackJob> hj(nq);
    std::vector<u32> sbeg, scnt;
    u64 M = 0, N = 0;
    u32 wtab_total = 0, rounds = 0, kmax = 0;
    for (size_t i = 0; i < nq; i++) {
        const Graph &g = *graphs[first + i];
        const QuerySpec &q = specs[first + i];
        hg[i] = {g.d_src, g.d_dst, g.d_time, g.d_color, M, g.m, (u32)N, g.n};
        PackQuery &Q = hq[i];
        Q.filter = q.filter();
        Q.keys = make_keys(mix64(q.seed + TM_GOLDEN));  // repeat 0
        Q.slot_off = (u32)sbeg.size();
        Q.wtab_off = wtab_total;
        Q.npts = 1u << q.k;
        Q.k = q.k;
        std::vector<u32> c(g.num_colors, 0);
        for (u32 col : q.multiset) c[col]++;
        for (u32 col = 0, off = 0; col < g.num_colors; col++) {
            sbeg.push_back(off);
            scnt.push_back(c[col]);
            off += c[col];
        }
        hj[i] = {Q.keys.ky, (u32)N, q.k, q.start == TMOTIF_ANY ? NONE : q.start + (u32)N,
                 q.end == TMOTIF_ANY ? NONE : q.end + (u32)N};
        wtab_total += q.k * PL;
        rounds = std::max(rounds, (Q.npts + PL - 1) / PL);
        kmax = std::max(kmax, q.k);
        M += g.m;
        N += g.n;
    }
    if (N >= NONE || M >= NONE) return fail(TMOTIF_ERR_UNSUPPORTED, "pack too large");
    TM_TRY(B.graphs.reserve(nq * sizeof(PackGraph)));
    TM_TRY(B.queries.reserve(nq * sizeof(PackQuery)));
    TM_TRY(B.jobs.reserve(nq * sizeof(PackJob)));
    TM_TRY(B.slot_begin.reserve(std::max<size_t>(sbeg.size(), 1) * 4));
    TM_TRY(B.slot_count.reserve(std::max<size_t>(scnt.size(), 1) * 4));
    TM_CUDA(cudaMemcpyAsync(B.graphs.p, hg.data(), nq * sizeof(PackGraph), cudaMemcpyHostToDevice, st));
    TM_CUDA(cudaMemcpyAsync(B.queries.p, hq.data(), nq * sizeof(PackQuery), cudaMemcpyHostToDevice, st));
    TM_CUDA(cudaMemcpyAsync(B.jobs.p, hj.data(), nq * sizeof(PackJob), cudaMemcpyHostToDevice, st));
    TM_CUDA(cudaMemcpyAsync(B.slot_begin.p, sbeg.data(), sbeg.size() * 4, cudaMemcpyHostToDevice, st));
    TM_CUDA(cudaMemcpyAsync(B.slot_count.p, scnt.data(), scnt.size() * 4, cudaMemcpyHostToDevice, st));
    // packed arcs and vertices
    TM_TRY(B.P_src.reserve(std::max<u64>(M, 1) * 4));
    TM_TRY(B.P_dst.reserve(std::max<u64>(M, 1) * 4));
    TM_TRY(B.P_time.reserve(std::max<u64>(M, 1) * 4));
    TM_TRY(B.P_color.reserve(std::max<u64>(N, 1) * 4));
    TM_TRY(B.jv.reserve(std::max<u64>(N, 1) * 4));
    k_pack_gather<<<(unsigned)nq, 256, 0, st>>>(B.graphs.as<PackGraph>(), B.P_src.as<u32>(), B.P_dst.as<u32>(),
                                                B.P_time.as<u32>(), B.P_color.as<u32>(), B.jv.as<u32>());
    TM_CUDA(cudaGetLastError());
    (*launches)++;
    TM_TRY(B.vflag.reserve(std::max<u64>(N, 1)));
    TM_TRY(B.act.reserve((N + 1) * 4));
    TM_TRY(B.act_list.reserve(std::max<u64>(N, 1) * 4));
    TM_TRY(B.keep.reserve((M + 1) * 4));
    TM_TRY(B.seg_lo.reserve(std::max<u64>(N, 1) * 4));
    TM_TRY(B.seg_hi.reserve(std::max<u64>(N, 1) * 4));
    TM_TRY(B.counters.reserve(64));
    TM_TRY(B.wtab.reserve((u64)wtab_total * 8));
    TM_TRY(B.out.reserve(nq * PL * 8));
    u32 *d_cnt = B.counters.as<u32>();
    u32 *h_cnt = (u32 *)pinned;
    // arcs the rounds filter: all packed arcs, then the previous round's kept
    // arcs (a later round keeps a subset: its queries are a subset)
    const u32 *c_src = B.P_src.as<u32>(), *c_dst = B.P_dst.as<u32>(), *c_time = B.P_time.as<u32>();
    u64 Mc = M;
    for (u32 r = 0; r < rounds; r++) {
        const u32 p0 = r * PL;
        DevBuf &o_src = (r & 1) ? B.g_src : B.f_src, &o_dst = (r & 1) ? B.g_dst : B.f_dst,
               &o_time = (r & 1) ? B.g_time : B.f_time;
        // filter: vertices with a query colour (queries with points in this
        // round), arcs between them inside their query's window
        k_pack_vflag<<<blocks_of(N + 1, 256), 256, 0, st>>>((u32)N, B.P_color.as<u32>(), B.jv.as<u32>(),
                                                           B.queries.as<PackQuery>(), B.slot_count.as<u32>(), p0,
                                                           B.vflag.as<uint8_t>(), B.act.as<u32>());
        k_pack_keep<<<blocks_of(Mc + 1, 256), 256, 0, st>>>(Mc, c_src, c_dst, c_time, B.vflag.as<uint8_t>(),
                                                           B.jv.as<u32>(), B.queries.as<PackQuery>(), B.keep.as<u32>());
        TM_CUDA(cudaGetLastError());
        TM_TRY(exclusive_scan_on(st, B.block_sums, B.keep.as<u32>(), Mc + 1, d_cnt + 0, launches));
        TM_TRY(exclusive_scan_on(st, B.block_sums, B.act.as<u32>(), N + 1, d_cnt + 2, launches));
        k_active_list<<<blocks_of(N, 256), 256, 0, st>>>((u32)N, B.act.as<u32>(), B.act_list.as<u32>());
        *launches += 3;
        TM_CUDA(cudaMemcpyAsync(h_cnt, d_cnt, 12, cudaMemcpyDeviceToHost, st));
        TM_CUDA(cudaStreamSynchronize(st));
        const u64 mf = h_cnt[0], n_act = h_cnt[2];
        TM_CUDA(cudaMemsetAsync(B.out.p, 0, nq * PL * 8, st));
        if (mf > 0) {
            TM_TRY(o_src.reserve(mf * 4));
            TM_TRY(o_dst.reserve(mf * 4));
            TM_TRY(o_time.reserve(mf * 4));
            TM_TRY(B.pos.reserve(mf * 4));
            TM_TRY(B.mark.reserve((mf + 1) * 4));
            TM_TRY(B.cp_in.reserve(mf * 4));
            TM_TRY(B.cp_out.reserve(mf * 4));
            k_compact<<<blocks_of(Mc, 256), 256, 0, st>>>(Mc, c_src, c_dst, c_time, B.keep.as<u32>(), o_src.as<u32>(),
                                                          o_dst.as<u32>(), o_time.as<u32>());
            TM_CUDA(cudaMemsetAsync(B.seg_lo.p, 0, N * 4, st));
            TM_CUDA(cudaMemsetAsync(B.seg_hi.p, 0, N * 4, st));
            TM_CUDA(cudaMemsetAsync(B.mark.p, 0, (mf + 1) * 4, st));
            k_segments<<<blocks_of(mf, 256), 256, 0, st>>>(mf, o_dst.as<u32>(), B.seg_lo.as<u32>(),
                                                           B.seg_hi.as<u32>(), (u32)N);
            k_pos<<<blocks_of(mf, 256), 256, 0, st>>>(mf, o_src.as<u32>(), o_time.as<u32>(), B.seg_lo.as<u32>(),
                                                      B.seg_hi.as<u32>(), B.pos.as<u32>(), B.mark.as<u32>(), (u32)N);
            TM_CUDA(cudaGetLastError());
            TM_TRY(exclusive_scan_on(st, B.block_sums, B.mark.as<u32>(), mf + 1, d_cnt + 1, launches));
            k_checkpoints<<<blocks_of(mf, 256), 256, 0, st>>>(mf, B.pos.as<u32>(), B.mark.as<u32>(),
                                                              B.cp_in.as<u32>(), B.cp_out.as<u32>(), nullptr, nullptr,
                                                              nullptr, nullptr, nullptr);
            TM_CUDA(cudaGetLastError());
            *launches += 4;
            TM_CUDA(cudaMemcpyAsync(h_cnt + 1, d_cnt + 1, 4, cudaMemcpyDeviceToHost, st));
            TM_CUDA(cudaStreamSynchronize(st));
            const u64 ncp = std::max<u32>(h_cnt[1], 1);
            TM_TRY(B.x.reserve(std::max<u64>(N, 1) * PL * 8));
            TM_TRY(B.C0.reserve(ncp * PL * 8));
            TM_TRY(B.C1.reserve(ncp * PL * 8));
            // coefficients of this round's points
            k_pack_wtab<<<(unsigned)nq, 128, 0, st>>>((u32)nq, B.queries.as<PackQuery>(), p0, B.wtab.as<u64>());
            if (n_act)
                k_pack_coef<<<(unsigned)((n_act + 7) / 8), 256, 0, st>>>(
                    (u32)n_act, B.act_list.as<u32>(), B.P_color.as<u32>(), B.jv.as<u32>(), B.queries.as<PackQuery>(),
                    B.graphs.as<PackGraph>(), B.slot_begin.as<u32>(), B.slot_count.as<u32>(), B.wtab.as<u64>(),
                    B.x.as<u64>());
            TM_CUDA(cudaGetLastError());
            *launches += 2;
            // layers 2..kmax: each segment follows its own query's k
            LayerParams lp{};  // every member zero or null
            lp.src = o_src.as<u32>();
            lp.dst = o_dst.as<u32>();
            lp.time = o_time.as<u32>();
            lp.cp_in = B.cp_in.as<u32>();
            lp.cp_out = B.cp_out.as<u32>();
            lp.seg_hi = B.seg_hi.as<u32>();
            lp.x = B.x.as<u64>();
            lp.m_f = mf;
            lp.n_chunks = (mf + PCHUNK - 1) / PCHUNK;
            lp.L = PL;
            lp.lane_groups = 1;
            lp.chunk = PCHUNK;
            lp.k = kmax;
            lp.start = lp.end = NONE;
            lp.T = 32;
            lp.jv = B.jv.as<u32>();
            lp.pjobs = B.jobs.as<PackJob>();
            lp.pout = B.out.as<u64>();
            u64 *bufs[2] = {B.C0.as<u64>(), B.C1.as<u64>()};
            const size_t smem = 8 * 256 * 8 + 2048;  // 18 KB: within the default dynamic limit
            TM_TRY(B.queue.reserve(sizeof(unsigned long long)));
            lp.queue = B.queue.as<unsigned long long>();
            lp.n_vert = (u32)N;
            lp.n_cp = ncp;
            TM_TRY(status_word(&lp.status));
            static const int per_sm = [&] {
                int nb = 0;
                const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pack_layer, 256, smem);
                return (e == cudaSuccess && nb > 0) ? nb : 1;
            }();
            const unsigned grid = (unsigned)std::min<u64>(blocks_of(lp.n_chunks, 8), (u64)per_sm * sm_count());
            for (u32 ell = 2; ell <= kmax; ell++) {
                lp.ell = ell;
                lp.Cin = bufs[ell & 1];
                lp.Cout = bufs[(ell + 1) & 1];
                TM_CUDA(cudaMemsetAsync(lp.queue, 0, sizeof(unsigned long long), st));
                k_pack_layer<<<grid, 256, smem, st>>>(lp);
                TM_CUDA(cudaGetLastError());
                (*launches)++;
            }
        }
        c_src = o_src.as<u32>();
        c_dst = o_dst.as<u32>();
        c_time = o_time.as<u32>();
        Mc = mf;
        TM_CUDA(cudaMemcpyAsync((char *)pinned + 64, B.out.p, nq * PL * 8, cudaMemcpyDeviceToHost, st));
        TM_CUDA(cudaStreamSynchronize(st));
        const u64 *h_out = (const u64 *)((const char *)pinned + 64);
        for (size_t i = 0; i < nq; i++) {
            const u32 npts = hq[i].npts;
            if (p0 >= npts) continue;
            std::vector<u64> &v = (*vals)[first + i];
            for (u32 lane = 0; lane < PL && p0 + lane < npts; lane++) v[p0 + lane] = h_out[i * PL + lane];
        }
    }
    return Status();
}

}  // namespace

bool pack_eligible(const QuerySpec &q)
{
    return q.repeats == 1 && q.p_begin == 0 && q.p_end == (1ull << q.k) && !(q.flags & TMOTIF_PREPROCESS_STATIC);
}

Status pack_decide(Graph *const *graphs, const QuerySpec *specs, size_t count, cudaStream_t st,
                   std::vector<std::vector<u64>> *vals, u64 *launches)
{
    vals->assign(count, std::vector<u64>());
    size_t max_q = 0;
    for (size_t i = 0; i < count; i++) (*vals)[i].assign(1ull << specs[i].k, 0);
    PackBuffers B;
    B.set_stream(st);
    // packs of consecutive queries up to PACK_ARCS arcs
    std::vector<std::pair<size_t, size_t>> packs;
    for (size_t i = 0; i < count;) {
        size_t j = i;
        u64 m = 0, n = 0;
        while (j < count && (j == i || (m + graphs[j]->m <= PACK_ARCS && n + graphs[j]->n < NONE / 2))) {
            m += graphs[j]->m;
            n += graphs[j]->n;
            j++;
        }
        packs.push_back({i, j});
        max_q = std::max(max_q, j - i);
        i = j;
    }
    void *pinned = nullptr;
    TM_CUDA(cudaMallocHost(&pinned, 64 + max_q * PL * 8));
    Status s;
    for (auto &pk : packs) {
        s = run_pack(graphs, specs, pk.first, pk.second, st, B, pinned, vals, launches);
        if (!s.ok()) break;
    }
    cudaFreeHost(pinned);
    B.release();
    return s;
}

}  // namespace tmo
