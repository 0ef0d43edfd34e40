// static.cu -- static-graph preprocessing sieve (Sec. 8.1 (ii), with the
// static generating function eq. gen-polynomial:1).
//
// The temporal graph is merged into the static graph E_s = {(a, b) : some arc
// a -> b at any time}, built once per resident graph and kept as two sorted
// pair lists: by (b, a) for the forward pass and by (a, b) for the backward
// pass.  Per query, a vertex u is kept iff it lies on a static path whose
// colours are M (first vertex = start, last = end when given).  Per sieve
// point A:
//   F_1(u) = x_u [u start-ok],  F_l(u) = x_u sum_{(v,u)} yf(v->u, l-1) F_{l-1}(v),
//   B_1(u) = [u end-ok],        B_l(u) = sum_{(u,w)} yb(u->w, k-l+1) x_w B_{l-1}(w),
//   Q_u^A  = sum_{r=1..k} F_r(u) B_{k-r+1}(u),
// and Q_u = sum_A Q_u^A.  Every term is the monomial of a whole walk of k
// vertices with u at position r (the arc from position p to p+1 carries yf
// before u and yb from u on), so Q_u != 0 (up to the sieve's one-sided error)
// iff some such walk is a matching path.  Every temporal path is a static
// path, so deleting the other vertices keeps every temporal match.
//   yf(a->b, p) = mix64(mix64(kf ^ (a << 32 | b)) ^ p), kf = mix64(qs ^ 0x4444..44),
//   yb(a->b, p) = mix64(mix64(kb ^ (a << 32 | b)) ^ p), kb = mix64(qs ^ 0x5555..55),
// qs the query seed of repeat 0; x_u^A as in the temporal sieve.
//
// A layer is one pass over the pair list sorted by owner (the gathering
// vertex): a warp takes a fixed chunk of pairs, accumulates y * In[other] per
// lane while the owner stays the same and XORs the run into Out[owner]
// atomically, so a vertex of any degree is split across warps.
#include <algorithm>

#include "gf64.cuh"
#include "internal.h"
#include "scan.cuh"

namespace tmo {

// per-query kernels of the temporal sieve (sieve.cu) reused here: vertex
// flags, the active-vertex list and the coefficients x_u^A
__global__ void k_vflag(u32 n, const u32 *color, const u32 *slot_count, const uint8_t *alive, uint8_t *vflag,
                        u32 *act);
__global__ void k_active_list(u32 n, const u32 *act, u32 *list);
__global__ void k_wtab(u32 k, u32 L, u64 p0, QueryKeys keys, u64 *wtab);
__global__ void __launch_bounds__(256) k_coef(u32 n_act, const u32 *list, u32 L, const u32 *color,
                                              const u32 *slot_begin, const u32 *slot_count, QueryKeys keys,
                                              const u64 *wtab, u64 *x, u32 n, u32 num_colors, u32 k);

namespace {

const u64 TAG_YF = 0x4444444444444444ull;
const u64 TAG_YB = 0x5555555555555555ull;
const u32 S_CHUNK = 64;        // most pairs per warp in a static layer
const u32 S_WARPS_PER_SM = 32;  // warps per SM a static layer aims to start

unsigned grid_of(u64 items, int threads) { return (unsigned)std::max<u64>(1, (items + threads - 1) / threads); }

__global__ void k_pair_keys(u64 m, const u32 *hi, const u32 *lo, int sb, u64 *keys)
{
    const u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m) keys[e] = ((u64)hi[e] << sb) | lo[e];
}

// flag[i] = 1 for the first copy of each key (keys sorted); flag[N] = 0.
__global__ void k_pair_unique(const u64 *keys, u64 N, u32 *flag)
{
    const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > N) return;
    if (i == N) { flag[N] = 0; return; }
    flag[i] = (i == 0 || keys[i - 1] != keys[i]) ? 1u : 0u;
}

// Unpack kept keys hi << sb | lo into owner (hi) and other (lo) arrays.
__global__ void k_pair_unpack(const u64 *keys, u64 N, const u32 *off, int sb, u32 *hi, u32 *lo)
{
    const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const u32 o = off ? off[i] : (u32)i;
    if (off && off[i + 1] == o) return;
    hi[o] = (u32)(keys[i] >> sb);
    lo[o] = (u32)(keys[i] & ((1ull << sb) - 1));
}

// Pairs whose two vertices carry a query colour (and are alive).
__global__ void k_pair_keep(u64 N, const u32 *own, const u32 *oth, const uint8_t *vflag, u32 *keep)
{
    const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > N) return;
    if (i == N) { keep[N] = 0; return; }
    keep[i] = (vflag[own[i]] && vflag[oth[i]]) ? 1u : 0u;
}

__global__ void k_pair_compact(u64 N, const u32 *own, const u32 *oth, const u32 *off, u32 *f_own, u32 *f_oth)
{
    const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const u32 o = off[i];
    if (off[i + 1] != o) {
        f_own[o] = own[i];
        f_oth[o] = oth[i];
    }
}

// One static layer: Out[own] ^= sum over the owner's pairs of y * In[oth]
// (per lane), In read through the base-case restriction `only` (vertex id
// or TMOTIF_ANY) when `base` is set.  y = mix64(mix64(key ^ (a << 32 | b)) ^ p)
// with (a, b) = (oth, own) when fwd, (own, oth) otherwise.  One warp per
// chunk of S pairs (S chosen by the launcher so that the launch fills the
// GPU), lanes tt and tt + 32 per thread; each batch of 32 pairs is loaded and
// its y computed once, one pair per thread, then broadcast by shuffles; with
// TAB the warp builds the nibble table of y (2 KB) and each lane product is
// 16 lookups.  A run of pairs with the same owner is flushed with one
// atomicXor per lane, so owners split across warps stay exact.
template <bool TAB>
__global__ void __launch_bounds__(256) k_static_layer(u64 M, u32 S, const u32 *own, const u32 *oth, u32 L,
                                                      const u64 *In, u64 *Out, u64 key, u32 p, int fwd, int base,
                                                      u32 only)
{
    __shared__ __align__(2048) u64 tabs[TAB ? 8 : 1][TAB ? 256 : 1];  // tables on 2 KB boundaries
    u64 *tab = tabs[TAB ? (threadIdx.x >> 5) : 0];
    const int tt = threadIdx.x & 31;
    const u64 w = (u64)blockIdx.x * 8 + (threadIdx.x >> 5);
    const u64 e0 = w * S;
    if (e0 >= M) return;  // whole warp leaves together
    const u64 e1 = min(M, e0 + S);
    const bool l0 = (u32)tt < L, l1 = (u32)tt + 32 < L;
    u64 a0 = 0, a1 = 0;
    u32 cur = own[e0];
    for (u64 eb = e0; eb < e1; eb += 32) {
        const u64 e = eb + tt;
        u32 o = 0, g = 0;
        u64 y = 0;
        if (e < e1) {
            o = own[e];
            g = oth[e];
            const u64 pair = fwd ? (((u64)g << 32) | o) : (((u64)o << 32) | g);
            y = mix64(mix64(key ^ pair) ^ (u64)p);
        }
        const int cnt = (int)min((u64)32, e1 - eb);
        for (int j = 0; j < cnt; j++) {
            const u32 oj = __shfl_sync(0xffffffffu, o, j), gj = __shfl_sync(0xffffffffu, g, j);
            const u64 yj = __shfl_sync(0xffffffffu, y, j);
            if (oj != cur) {
                if (l0 && a0) atomicXor(&Out[(u64)cur * L + tt], a0);
                if (l1 && a1) atomicXor(&Out[(u64)cur * L + tt + 32], a1);
                a0 = a1 = 0;
                cur = oj;
            }
            const bool use = !base || only == TMOTIF_ANY || only == gj;
            const u64 v0 = (l0 && use) ? In[(u64)gj * L + tt] : 0;
            const u64 v1 = (l1 && use) ? In[(u64)gj * L + tt + 32] : 0;
            if (TAB) {
                __syncwarp();
                gf_table_build(tab, yj, tt, 32);
                __syncwarp();
                a0 ^= gf_table_mul(tab, v0);
                a1 ^= gf_table_mul(tab, v1);
            } else {
                a0 ^= gf_mul(yj, v0);
                a1 ^= gf_mul(yj, v1);
            }
        }
    }
    if (l0 && a0) atomicXor(&Out[(u64)cur * L + tt], a0);
    if (l1 && a1) atomicXor(&Out[(u64)cur * L + tt + 32], a1);
}

// Out[u] = x_u * In[u] per lane for the active vertices.
__global__ void k_static_scale(u64 n_act, const u32 *list, u32 L, const u64 *x, const u64 *In, u64 *Out)
{
    const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_act * L) return;
    const u64 r = (u64)list[i / L] * L + (i % L);
    Out[r] = gf_mul(x[r], In[r]);
}

// Q_u ^= sum over lanes of sum_{r=1..k} F_r(u) B_{k-r+1}(u) for the active
// vertices (one warp per vertex).  F[l], B[l] (l = 2..k) are n x L arrays;
// F_1 = x [start-ok], B_1 = [end-ok].
struct StaticArrays {
    const u64 *F[TMOTIF_KMAX + 1];
    const u64 *B[TMOTIF_KMAX + 1];
};

__global__ void __launch_bounds__(256) k_static_combine(u64 n_act, const u32 *list, u32 L, u32 k, StaticArrays A,
                                                        const u64 *x, u32 start, u32 end, u64 *Qv)
{
    const int tt = threadIdx.x & 31;
    const u64 v = (u64)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (v >= n_act) return;
    const u32 u = list[v];
    const bool s_ok = start == TMOTIF_ANY || start == u, e_ok = end == TMOTIF_ANY || end == u;
    u64 q = 0;
    for (u32 lane = tt; lane < L; lane += 32) {
        const u64 r = (u64)u * L + lane;
        const u64 f1 = s_ok ? x[r] : 0;
        u64 s = gf_mul(f1, A.B[k][r]);
        for (u32 l = 2; l < k; l++) s ^= gf_mul(A.F[l][r], A.B[k - l + 1][r]);
        if (e_ok) s ^= A.F[k][r];
        q ^= s;
    }
    for (int o = 16; o > 0; o >>= 1) q ^= __shfl_xor_sync(0xffffffffu, q, o);
    if (tt == 0) Qv[u] ^= q;
}

__global__ void k_static_mask(u32 n, const u64 *Qv, uint8_t *mask)
{
    const u64 u = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n) mask[u] = Qv[u] ? 1 : 0;
}

template <bool TAB>
Status launch_static_layer(cudaStream_t st, u64 M, const u32 *own, const u32 *oth, u32 L, const u64 *In, u64 *Out,
                           u64 key, u32 p, int fwd, int base, u32 only)
{
    if (M == 0) return Status();
    // pairs per warp: enough warps for every SM to hold S_WARPS_PER_SM of
    // them, at most S_CHUNK pairs per warp
    const u64 target = (u64)sm_count() * S_WARPS_PER_SM;
    const u32 S = (u32)std::min<u64>(S_CHUNK, std::max<u64>(1, (M + target - 1) / target));
    const u64 warps = (M + S - 1) / S;
    k_static_layer<TAB><<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(M, S, own, oth, L, In, Out, key, p, fwd, base,
                                                                    only);
    TM_CUDA(cudaGetLastError());
    return Status();
}

}  // namespace

// E_s of a resident graph, built once (two radix sorts of packed pairs).
Status static_graph_ensure(Graph &g)
{
    if (g.s_built) return Status();
    cudaStream_t st = g.stream;
    const u64 m = g.m;
    int sb = 1;
    while (sb < 32 && ((u64)(g.n > 0 ? g.n - 1 : 0) >> sb)) sb++;
    DevBuf k1, k2, flag, cnt;
    k1.stream = k2.stream = flag.stream = cnt.stream = st;
    TM_TRY(k1.reserve(std::max<u64>(m, 1) * 8));
    TM_TRY(k2.reserve(std::max<u64>(m, 1) * 8));
    TM_TRY(flag.reserve((m + 1) * 4));
    TM_TRY(cnt.reserve(16));
    u64 launches = 0;
    u64 ms = 0;
    if (m) {
        // by (dst, src): pairs (a -> b) keyed b << sb | a, deduplicated
        k_pair_keys<<<grid_of(m, 256), 256, 0, st>>>(m, g.d_dst, g.d_src, sb, k1.as<u64>());
        u64 *sorted = nullptr;
        TM_TRY(radix_sort_u64(st, k1.as<u64>(), k2.as<u64>(), m, 2 * sb, cnt.as<u32>(), &sorted, &launches));
        k_pair_unique<<<grid_of(m + 1, 256), 256, 0, st>>>(sorted, m, flag.as<u32>());
        TM_TRY(exclusive_scan_on(st, g.ws.block_sums, flag.as<u32>(), m + 1, cnt.as<u32>(), &launches));
        u32 h = 0;
        TM_CUDA(cudaMemcpyAsync(&h, cnt.p, 4, cudaMemcpyDeviceToHost, st));
        TM_CUDA(cudaStreamSynchronize(st));
        ms = h;
        TM_TRY(dev_alloc((void **)&g.s_in, std::max<u64>(ms, 1) * 8, st));
        TM_TRY(dev_alloc((void **)&g.s_out, std::max<u64>(ms, 1) * 8, st));
        // s_in = [dst (owner) | src], s_out = [src (owner) | dst]
        k_pair_unpack<<<grid_of(m, 256), 256, 0, st>>>(sorted, m, flag.as<u32>(), sb, g.s_in, g.s_in + ms);
        u64 *other = (sorted == k1.as<u64>()) ? k2.as<u64>() : k1.as<u64>();
        k_pair_keys<<<grid_of(ms, 256), 256, 0, st>>>(ms, g.s_in + ms, g.s_in, sb, other);
        u64 *sorted2 = nullptr;
        TM_TRY(radix_sort_u64(st, other, sorted, ms, 2 * sb, cnt.as<u32>(), &sorted2, &launches));
        k_pair_unpack<<<grid_of(ms, 256), 256, 0, st>>>(sorted2, ms, nullptr, sb, g.s_out, g.s_out + ms);
        TM_CUDA(cudaGetLastError());
        TM_CUDA(cudaStreamSynchronize(st));
    }
    g.m_static = ms;
    g.s_built = true;
    g.resident_bytes += ms * 16;
    g.prof.stats.launches += launches + 5;
    k1.release();
    k2.release();
    flag.release();
    cnt.release();
    return Status();
}

Status static_sieve(Graph &g, const QuerySpec &q, const uint8_t *d_alive, u64 *d_Qv, u64 *kept_pairs)
{
    TM_TRY(static_graph_ensure(g));
    cudaStream_t st = g.stream;
    Workspace &w = g.ws;
    StaticWork &sw = g.sw;
    sw.set_stream(st);
    const u32 n = g.n, k = q.k;
    u64 *launches = (u64 *)&g.prof.stats.launches;
    TM_CUDA(cudaMemsetAsync(d_Qv, 0, (u64)std::max<u32>(n, 1) * 8, st));
    if (kept_pairs) *kept_pairs = 0;

    // query colours -> slots; vertex flags and the active list
    std::vector<u32> sbeg(g.num_colors, 0), scnt(g.num_colors, 0);
    for (u32 c : q.multiset) scnt[c]++;
    for (u32 c = 0, off = 0; c < g.num_colors; c++) { sbeg[c] = off; off += scnt[c]; }
    TM_TRY(w.slot_begin.reserve(g.num_colors * 4));
    TM_TRY(w.slot_count.reserve(g.num_colors * 4));
    TM_TRY(w.counters.reserve(64));
    TM_TRY(w.vflag.reserve(std::max<u64>(n, 1)));
    TM_TRY(w.act.reserve(((u64)n + 1) * 4));
    TM_TRY(w.act_list.reserve(std::max<u64>(n, 1) * 4));
    TM_CUDA(cudaMemcpyAsync(w.slot_begin.p, sbeg.data(), g.num_colors * 4, cudaMemcpyHostToDevice, st));
    TM_CUDA(cudaMemcpyAsync(w.slot_count.p, scnt.data(), g.num_colors * 4, cudaMemcpyHostToDevice, st));
    u32 *d_cnt = w.counters.as<u32>();
    k_vflag<<<grid_of((u64)n + 1, 256), 256, 0, st>>>(n, g.d_color, w.slot_count.as<u32>(), d_alive,
                                                      w.vflag.as<uint8_t>(), w.act.as<u32>());
    TM_TRY(exclusive_scan_on(st, w.block_sums, w.act.as<u32>(), (u64)n + 1, d_cnt + 2, launches));
    k_active_list<<<grid_of(n, 256), 256, 0, st>>>(n, w.act.as<u32>(), w.act_list.as<u32>());
    // pairs among flagged vertices, in both orders
    const u64 ms = g.m_static;
    TM_TRY(sw.keep.reserve((ms + 1) * 4));
    TM_TRY(sw.in.reserve(std::max<u64>(ms, 1) * 8));
    TM_TRY(sw.out.reserve(std::max<u64>(ms, 1) * 8));
    for (int pass = 0; pass < 2 && ms; pass++) {
        const u32 *base = pass == 0 ? g.s_in : g.s_out;
        k_pair_keep<<<grid_of(ms + 1, 256), 256, 0, st>>>(ms, base, base + ms, w.vflag.as<uint8_t>(),
                                                         sw.keep.as<u32>());
        TM_TRY(exclusive_scan_on(st, w.block_sums, sw.keep.as<u32>(), ms + 1, d_cnt + 4 + pass, launches));
        u32 *dstp = pass == 0 ? sw.in.as<u32>() : sw.out.as<u32>();
        k_pair_compact<<<grid_of(ms, 256), 256, 0, st>>>(ms, base, base + ms, sw.keep.as<u32>(), dstp, dstp + ms);
        *launches += 2;
    }
    *launches += 2;
    TM_CUDA(cudaGetLastError());
    u32 hc[6] = {0, 0, 0, 0, 0, 0};
    TM_CUDA(cudaMemcpyAsync(hc, d_cnt, 24, cudaMemcpyDeviceToHost, st));
    TM_CUDA(cudaStreamSynchronize(st));
    const u64 n_act = hc[2], M = ms ? hc[4] : 0;
    if (kept_pairs) *kept_pairs = M;
    if (n_act == 0) return Status();
    // compacted lists: owner array at [0, M), other at [ms, ms + M)
    const u32 *in_own = sw.in.as<u32>(), *in_oth = sw.in.as<u32>() + ms;
    const u32 *out_own = sw.out.as<u32>(), *out_oth = sw.out.as<u32>() + ms;

    // lane width: as in the temporal sieve, halved while 2k+1 vertex arrays
    // of L lanes would not fit
    const u64 npts = 1ull << k;
    u32 L = 4;
    while (L < 64 && L < npts) L <<= 1;
    {
        size_t room = 0;
        TM_TRY(device_headroom(&room));
        room += sw.arrays.bytes + w.x.bytes;
        while (L > 4 && (u64)n * 8 * (2 * k + 2) * L > room / 10 * 9) L >>= 1;
    }
    const u64 row = (u64)n * L;  // u64 per vertex array
    // arrays: F[2..k], B[2..k], Bx ping-pong (2)
    TM_TRY(sw.arrays.reserve(std::max<u64>(row, 1) * 8 * (2 * (k - 1) + 2)));
    TM_TRY(w.x.reserve(std::max<u64>(row, 1) * 8));
    TM_TRY(w.wtab.reserve((u64)k * L * 8));
    u64 *arr = sw.arrays.as<u64>();
    StaticArrays A;
    u64 *F[TMOTIF_KMAX + 1] = {nullptr}, *B[TMOTIF_KMAX + 1] = {nullptr};
    for (u32 l = 2; l <= k; l++) {
        F[l] = arr + (u64)(l - 2) * row;
        B[l] = arr + (u64)(k - 1 + l - 2) * row;
        A.F[l] = F[l];
        A.B[l] = B[l];
    }
    u64 *Bx[2] = {arr + (u64)(2 * (k - 1)) * row, arr + (u64)(2 * (k - 1) + 1) * row};
    const u64 qs = mix64(q.seed + TM_GOLDEN);  // repeat 0
    const QueryKeys keys = make_keys(qs);
    const u64 kf = mix64(qs ^ TAG_YF), kb = mix64(qs ^ TAG_YB);
    const bool tab = L >= 32;
    auto layer = [&](u64 Mp, const u32 *own, const u32 *oth, const u64 *In, u64 *Out, u64 key, u32 p, int fwd,
                     int base, u32 only) -> Status {
        (*launches)++;
        cudaEvent_t ea = nullptr;
        TM_TRY(g.prof.begin(st, &ea));
        TM_TRY(tab ? launch_static_layer<true>(st, Mp, own, oth, L, In, Out, key, p, fwd, base, only)
                   : launch_static_layer<false>(st, Mp, own, oth, L, In, Out, key, p, fwd, base, only));
        TM_TRY(g.prof.end(st, ea, FAM_STATIC));
        tmotif_stats &sx = g.prof.stats;
        sx.static_launches++;
        sx.static_gf_muls += Mp * L;
        if (tab) {
            sx.static_table_muls += Mp * L;
            sx.static_table_builds += Mp;
        }
        return Status();
    };
    for (u64 p0 = 0; p0 < npts; p0 += L) {
        k_wtab<<<grid_of((u64)k * L, 128), 128, 0, st>>>(k, L, p0, keys, w.wtab.as<u64>());
        k_coef<<<(unsigned)((n_act + 7) / 8), 256, 0, st>>>((u32)n_act, w.act_list.as<u32>(), L, g.d_color,
                                                             w.slot_begin.as<u32>(), w.slot_count.as<u32>(), keys,
                                                             w.wtab.as<u64>(), w.x.as<u64>(), g.n, g.num_colors, k);
        TM_CUDA(cudaMemsetAsync(arr, 0, row * 8 * 2 * (k - 1), st));
        const u64 *x = w.x.as<u64>();
        const u32 *act = w.act_list.as<u32>();
        // forward: F_l = x * sum over in-pairs of yf * F_{l-1} (F_1 = x [start-ok])
        for (u32 l = 2; l <= k; l++) {
            TM_TRY(layer(M, in_own, in_oth, l == 2 ? x : F[l - 1], F[l], kf, l - 1, 1, l == 2, q.start));
            k_static_scale<<<grid_of(n_act * L, 256), 256, 0, st>>>(n_act, act, L, x, F[l], F[l]);
        }
        // backward: B_l = sum over out-pairs of yb * x_w B_{l-1}(w) (x B_1 = x [end-ok])
        for (u32 l = 2; l <= k; l++) {
            const u64 *in = l == 2 ? x : Bx[l & 1];
            TM_TRY(layer(M, out_own, out_oth, in, B[l], kb, k - l + 1, 0, l == 2, q.end));
            if (l < k) k_static_scale<<<grid_of(n_act * L, 256), 256, 0, st>>>(n_act, act, L, x, B[l], Bx[(l + 1) & 1]);
        }
        k_static_combine<<<(unsigned)((n_act + 7) / 8), 256, 0, st>>>(n_act, act, L, k, A, x, q.start, q.end, d_Qv);
        *launches += 3 + 2 * (k - 1);
        TM_CUDA(cudaGetLastError());
    }
    return Status();
}

Status static_mask(Graph &g, const QuerySpec &q, const uint8_t *d_alive, uint8_t *d_mask, u64 *kept_pairs)
{
    StaticWork &sw = g.sw;
    sw.set_stream(g.stream);
    TM_TRY(sw.qv.reserve(std::max<u64>(g.n, 1) * 8));
    TM_TRY(static_sieve(g, q, d_alive, sw.qv.as<u64>(), kept_pairs));
    k_static_mask<<<grid_of(g.n, 256), 256, 0, g.stream>>>(g.n, sw.qv.as<u64>(), d_mask);
    g.prof.stats.launches++;
    TM_CUDA(cudaGetLastError());
    return Status();
}

void StaticWork::set_stream(cudaStream_t s)
{
    DevBuf *all[] = {&keep, &in, &out, &arrays, &qv, &mask};
    for (DevBuf *b : all) b->stream = s;
}

void StaticWork::release()
{
    DevBuf *all[] = {&keep, &in, &out, &arrays, &qv, &mask};
    for (DevBuf *b : all) b->release();
}

}  // namespace tmo
