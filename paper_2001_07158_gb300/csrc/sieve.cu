// sieve.cu -- per-query kernels of the constrained multilinear sieve.
//
// For one query the device runs, per lane batch of L sieve points:
//   1. prep (once per query): keep the arcs whose endpoints carry a query
//      colour and whose time is in the window (Sec. 7.1 preprocessing (i):
//      vertices whose colour is not in M contribute x_u = 0), compact them in
//      (dst, time, src) order, find for every arc e = (a -> b, t) the last
//      in-arc of a with time < t ("pos"), and number the distinct pos values
//      ("checkpoints": the only prefix values any later arc reads);
//   2. coefficients x_u^A = sum_{d in S_c(u)} v_{u,d} W_d^A (Lemma 5.5,
//      eq. motif:1) for every lane;
//   3. layers l = 2..k of eq. (gen-polynomial:3), edge-centric: for arc e into
//      b, H_l[e] = y_{e,l-1} * P_{a,l-1,t(e)-1}; P_{b,l,i} is x_b times the XOR
//      of H_l over b's in-arcs with time <= i (the "+ P_{u,l,i-1}" stay term
//      is the running prefix); it is stored only at checkpoints; the last
//      layer XORs x_b * (sum of H_k over b's in-arcs) into the lane's sum.
// P_{a,1,i} = x_a for all i (the base case, read at i = 0 as well), so layer 2
// reads x directly.
#include <algorithm>
#include <cstring>

#include "gf64.cuh"
#include "internal.h"

namespace tmo {

// ---------------------------------------------------------------------------
// Exclusive scan of u32 arrays (three phases: tile sums, scan of tile sums,
// tile scan).  Totals fit in u32 because arc counts are < 2^32.
// ---------------------------------------------------------------------------
static const int SCAN_THREADS = 256;
static const int SCAN_PER_THREAD = 16;
static const int SCAN_TILE = SCAN_THREADS * SCAN_PER_THREAD;

__device__ __forceinline__ u32 block_exclusive_scan(u32 v, u32 *total)
{
    __shared__ u32 warp_sums[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    u32 x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        u32 y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        u32 s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            u32 y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) warp_sums[lane] = s;
    }
    __syncthreads();
    u32 before = (wid > 0 ? warp_sums[wid - 1] : 0) + x - v;
    if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_tile_sum(const u32 *in, u64 N, u32 *tile_sums)
{
    u64 base = (u64)blockIdx.x * SCAN_TILE + (u64)threadIdx.x * SCAN_PER_THREAD;
    u32 s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_PER_THREAD; i++)
        if (base + i < N) s += in[base + i];
    u32 tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

// One block: exclusive scan of ntiles values in place; total to *total.
__global__ void __launch_bounds__(1024) k_scan_tiles(u32 *sums, u32 ntiles, u32 *total)
{
    const u32 per = (ntiles + blockDim.x - 1) / blockDim.x;
    const u32 b = threadIdx.x * per, e = min(ntiles, b + per);
    u32 s = 0;
    for (u32 i = b; i < e; i++) s += sums[i];
    u32 tot;
    u32 run = block_exclusive_scan(s, &tot);
    for (u32 i = b; i < e; i++) {
        u32 v = sums[i];
        sums[i] = run;
        run += v;
    }
    if (threadIdx.x == 0) *total = tot;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_tile_scan(const u32 *in, u64 N, const u32 *tile_off, u32 *out)
{
    u64 base = (u64)blockIdx.x * SCAN_TILE + (u64)threadIdx.x * SCAN_PER_THREAD;
    u32 v[SCAN_PER_THREAD];
    u32 s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_PER_THREAD; i++) {
        v[i] = (base + i < N) ? in[base + i] : 0;
        s += v[i];
    }
    u32 run = block_exclusive_scan(s, nullptr) + tile_off[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_PER_THREAD; i++) {
        if (base + i < N) out[base + i] = run;
        run += v[i];
    }
}

// In-place exclusive scan of a[0..N); writes the total to d_total (device u32).
static Status exclusive_scan(Graph &g, u32 *a, u64 N, u32 *d_total)
{
    Workspace &w = g.ws;
    u64 ntiles = (N + SCAN_TILE - 1) / SCAN_TILE;
    if (ntiles == 0) ntiles = 1;
    TM_TRY(w.block_sums.reserve(ntiles * sizeof(u32)));
    u32 *sums = w.block_sums.as<u32>();
    k_tile_sum<<<(unsigned)ntiles, SCAN_THREADS, 0, g.stream>>>(a, N, sums);
    k_scan_tiles<<<1, 1024, 0, g.stream>>>(sums, (u32)ntiles, d_total);
    k_tile_scan<<<(unsigned)ntiles, SCAN_THREADS, 0, g.stream>>>(a, N, sums, a);
    g.prof.stats.launches += 3;
    TM_CUDA(cudaGetLastError());
    return Status();
}

// ---------------------------------------------------------------------------
// Per-query preparation
// ---------------------------------------------------------------------------
__global__ void k_vflag(u32 n, const u32 *color, const u32 *slot_count, const uint8_t *alive, uint8_t *vflag)
{
    u64 u = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    bool f = slot_count[color[u]] > 0;
    if (alive) f = f && alive[u];
    vflag[u] = f ? 1 : 0;
}

__global__ void k_keep(u64 m, const u32 *src, const u32 *dst, const u32 *time, const uint8_t *vflag, u32 t_min,
                       u32 t_max, u32 *keep)
{
    u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (e > m) return;
    if (e == m) { keep[m] = 0; return; }
    u32 t = time[e];
    bool k = vflag[src[e]] && vflag[dst[e]] && t >= t_min && (t_max == 0 || t <= t_max);
    keep[e] = k ? 1 : 0;
}

// keep[] holds exclusive offsets (length m+1); arc e is kept iff keep[e+1] > keep[e].
__global__ void k_compact(u64 m, const u32 *src, const u32 *dst, const u32 *time, const u32 *off, u32 *f_src,
                          u32 *f_dst, u32 *f_time)
{
    u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    u32 o = off[e];
    if (off[e + 1] != o) {
        f_src[o] = src[e];
        f_dst[o] = dst[e];
        f_time[o] = time[e];
    }
}

// In-segment [seg_lo[v], seg_hi[v]) of each destination in the filtered arcs.
__global__ void k_segments(u64 mf, const u32 *f_dst, u32 *seg_lo, u32 *seg_hi)
{
    u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= mf) return;
    u32 d = f_dst[e];
    if (e == 0 || f_dst[e - 1] != d) seg_lo[d] = (u32)e;
    if (e + 1 == mf || f_dst[e + 1] != d) seg_hi[d] = (u32)(e + 1);
}

// pos[e] = last in-arc of src(e) with time < time(e) (strictly increasing times,
// Sec. 3), or NONE; marks that arc as a checkpoint.
__global__ void k_pos(u64 mf, const u32 *f_src, const u32 *f_time, const u32 *seg_lo, const u32 *seg_hi,
                      u32 *pos, u32 *mark)
{
    u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= mf) return;
    u32 a = f_src[e], t = f_time[e];
    u32 lo = seg_lo[a], hi = seg_hi[a];
    // first index in [lo, hi) with time >= t
    while (lo < hi) {
        u32 mid = lo + ((hi - lo) >> 1);
        if (f_time[mid] < t) lo = mid + 1;
        else hi = mid;
    }
    u32 p = NONE;
    if (lo > seg_lo[a]) {
        p = lo - 1;
        mark[p] = 1;
    }
    pos[e] = p;
}

// mark[] holds exclusive checkpoint numbers (length mf+1).
__global__ void k_checkpoints(u64 mf, const u32 *pos, const u32 *ck, u32 *cp_in, u32 *cp_out)
{
    u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= mf) return;
    u32 p = pos[e];
    cp_in[e] = (p == NONE) ? NONE : ck[p];
    u32 c = ck[e];
    cp_out[e] = (ck[e + 1] != c) ? c : NONE;
}

// ---------------------------------------------------------------------------
// Coefficients (Lemma 5.5, eq. motif:1)
// ---------------------------------------------------------------------------
// W_d^A = sum_{j in A} w_{d,j} for slots d < k and lanes of the batch.
__global__ void k_wtab(u32 k, u32 L, u64 p0, QueryKeys keys, u64 *wtab)
{
    u32 i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k * L) return;
    u32 d = i / L, lane = i % L;
    u64 point = p0 + lane;
    u64 s = 0;
    for (u32 j = 0; j < k; j++)
        if ((point >> j) & 1u) s ^= coef_w(keys, d, j);
    wtab[i] = s;
}

// x_u^A = sum_{d in S_c(u)} v_{u,d} W_d^A, for vertices that carry a query colour.
__global__ void k_coef(u32 n, u32 L, const uint8_t *vflag, const u32 *color, const u32 *slot_begin,
                       const u32 *slot_count, QueryKeys keys, const u64 *wtab, u64 *x)
{
    u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (u64)n * L) return;
    u32 u = (u32)(i / L), lane = (u32)(i % L);
    if (!vflag[u]) return;
    u32 c = color[u];
    u32 d0 = slot_begin[c], d1 = d0 + slot_count[c];
    u64 s = 0;
    for (u32 d = d0; d < d1; d++) s ^= gf_mul(coef_v(keys, u, d), wtab[(u64)d * L + lane]);
    x[i] = s;
}

// ---------------------------------------------------------------------------
// Layer kernel: eq. (gen-polynomial:3), one walk length per launch.
// ---------------------------------------------------------------------------
struct LayerParams {
    const u32 *src, *dst, *time, *cp_in, *cp_out, *seg_hi;
    const u64 *x;
    const u64 *Cin;
    u64 *Cout;
    u64 *out;
    u64 m_f;
    u64 n_chunks;
    u64 ky;
    u32 L, lane_groups, chunk, ell, k, start, end;
};

// A team of T threads owns 2T consecutive lanes (16 bytes per thread) and walks
// one chunk of whole in-segments in arc order.  Segments are never split, so a
// running XOR is the prefix of eq. (3)'s stay term.  With TAB the team builds,
// per arc, the nibble table of y_{e,l-1} in shared memory and every lane's
// y-product is 16 table loads; x-products (one per checkpoint and per segment
// at the last layer) use the register multiply.
template <int T, bool TAB>
__global__ void __launch_bounds__(256) k_layer(LayerParams p)
{
    extern __shared__ __align__(16) u64 smem[];
    u64 *red = smem;
    u64 *tab = smem + ((p.L + 1u) & ~1u) + (size_t)(threadIdx.x / T) * 256;
    for (u32 i = threadIdx.x; i < p.L; i += blockDim.x) red[i] = 0;
    __syncthreads();

    const int tt = threadIdx.x % T;
    const u32 team_mask = (T == 32) ? 0xffffffffu : (((1u << T) - 1u) << (((threadIdx.x & 31) / T) * T));
    const u64 team = (u64)blockIdx.x * (blockDim.x / T) + threadIdx.x / T;
    const u64 chunk = team / p.lane_groups;
    const u32 lane0 = (u32)(team % p.lane_groups) * (2 * T) + 2 * tt;
    const u64 Lw = p.L;
    u64 q0 = 0, q1 = 0;

    if (chunk < p.n_chunks) {
        const u64 b0 = chunk * p.chunk;
        const u64 b1 = min(b0 + p.chunk, p.m_f);
        u64 begin = b0, stop = b1;
        if (b0 > 0 && p.dst[b0] == p.dst[b0 - 1]) begin = p.seg_hi[p.dst[b0]];
        if (b1 < p.m_f && p.dst[b1] == p.dst[b1 - 1]) stop = p.seg_hi[p.dst[b1]];

        u32 cur = NONE;
        u64 xc0 = 0, xc1 = 0, acc0 = 0, acc1 = 0;
        const bool last = (p.ell == p.k);
        for (u64 base = begin; base < stop; base += T) {
            const u64 e = base + tt;
            u32 s = 0, d = NONE, ci = NONE, co = NONE;
            u64 y = 0;
            if (e < stop) {
                s = p.src[e];
                d = p.dst[e];
                const u32 t = p.time[e];
                if (p.ell > 2) ci = p.cp_in[e];
                if (!last) co = p.cp_out[e];
                y = coef_y(mix64(p.ky ^ (((u64)s << 32) | d)), t, p.ell - 1);
            }
            const int cnt = (int)min((u64)T, stop - base);
            for (int j = 0; j < cnt; j++) {
                const u32 dj = __shfl_sync(team_mask, d, j, T);
                const u32 sj = __shfl_sync(team_mask, s, j, T);
                const u32 cij = __shfl_sync(team_mask, ci, j, T);
                const u32 coj = __shfl_sync(team_mask, co, j, T);
                const u64 yj = __shfl_sync(team_mask, y, j, T);
                if (dj != cur) {
                    if (last && cur != NONE && (p.end == NONE || cur == p.end)) {
                        q0 ^= gf_mul(xc0, acc0);
                        q1 ^= gf_mul(xc1, acc1);
                    }
                    cur = dj;
                    acc0 = acc1 = 0;
                    const ulonglong2 xv = *(const ulonglong2 *)(p.x + (u64)dj * Lw + lane0);
                    xc0 = xv.x;
                    xc1 = xv.y;
                }
                bool have = false;
                ulonglong2 in;
                if (p.ell == 2) {
                    if (p.start == NONE || sj == p.start) {
                        in = *(const ulonglong2 *)(p.x + (u64)sj * Lw + lane0);
                        have = true;
                    }
                } else if (cij != NONE) {
                    in = *(const ulonglong2 *)(p.Cin + (u64)cij * Lw + lane0);
                    have = true;
                }
                if (have) {  // uniform across the team
                    if (TAB) {
                        __syncwarp(team_mask);  // earlier lookups are done
                        gf_table_build(tab, yj, tt, T);
                        __syncwarp(team_mask);  // table complete
                        acc0 ^= gf_table_mul(tab, in.x);
                        acc1 ^= gf_table_mul(tab, in.y);
                    } else {
                        acc0 ^= gf_mul(yj, in.x);
                        acc1 ^= gf_mul(yj, in.y);
                    }
                }
                if (coj != NONE) {
                    ulonglong2 o;
                    o.x = gf_mul(xc0, acc0);
                    o.y = gf_mul(xc1, acc1);
                    *(ulonglong2 *)(p.Cout + (u64)coj * Lw + lane0) = o;
                }
            }
        }
        if (last && cur != NONE && (p.end == NONE || cur == p.end)) {
            q0 ^= gf_mul(xc0, acc0);
            q1 ^= gf_mul(xc1, acc1);
        }
    }
    if (p.ell == p.k) {
        if (q0) atomicXor(&red[lane0], q0);
        if (q1) atomicXor(&red[lane0 + 1], q1);
        __syncthreads();
        for (u32 i = threadIdx.x; i < p.L; i += blockDim.x)
            if (red[i]) atomicXor(&p.out[i], red[i]);
    }
}

// ---------------------------------------------------------------------------
// Diagnostic multiply kernel
// ---------------------------------------------------------------------------
__global__ void k_gf_mul(const u64 *a, const u64 *b, u64 *out, u64 n)
{
    u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = gf_mul(a[i], b[i]);
}

Status gf_mul_batch(const u64 *a, const u64 *b, u64 *out, u64 n)
{
    if (n == 0) return Status();
    u64 *d = nullptr;
    TM_CUDA(cudaMalloc(&d, 3 * n * sizeof(u64)));
    cudaError_t e = cudaMemcpy(d, a, n * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + n, b, n * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_gf_mul<<<(unsigned)((n + 255) / 256), 256>>>(d, d + n, d + 2 * n, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, d + 2 * n, n * 8, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "gf_mul_batch");
    return Status();
}

// ---------------------------------------------------------------------------
// Host orchestration of one decision.
// ---------------------------------------------------------------------------
static inline unsigned grid_for(u64 items, int threads) { return (unsigned)((items + threads - 1) / threads); }

template <int T, bool TAB>
static Status launch_layer_t(Graph &g, const LayerParams &lp, u64 teams)
{
    const int threads = 256;
    const u64 teams_per_block = threads / T;
    const unsigned blocks = (unsigned)((teams + teams_per_block - 1) / teams_per_block);
    const size_t smem = (((size_t)lp.L + 1) & ~(size_t)1) * sizeof(u64) + (TAB ? teams_per_block * 256 * 8 : 0);
    static bool attr_set = false;
    if (!attr_set) {
        TM_CUDA(cudaFuncSetAttribute(k_layer<T, TAB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
        attr_set = true;
    }
    k_layer<T, TAB><<<blocks, threads, smem, g.stream>>>(lp);
    return Status();
}

static Status launch_layer(Graph &g, const LayerParams &lp, int T, u64 teams)
{
    // L <= 64 lanes per batch, so the shared XOR buffer is at most 512 B; the
    // tables take 2 KB per team.
    switch (T) {
        case 2: TM_TRY((launch_layer_t<2, false>(g, lp, teams))); break;
        case 4: TM_TRY((launch_layer_t<4, false>(g, lp, teams))); break;
        case 8: TM_TRY((launch_layer_t<8, false>(g, lp, teams))); break;
        case 16: TM_TRY((launch_layer_t<16, false>(g, lp, teams))); break;
        default: TM_TRY((launch_layer_t<32, false>(g, lp, teams))); break;
    }
    g.prof.stats.launches++;
    g.prof.stats.layer_launches++;
    TM_CUDA(cudaGetLastError());
    return Status();
}

static const u32 LANES_MAX = 64;  // lanes per batch (one warp owns 64 lanes)

Status sieve_decide(Graph &g, const QuerySpec &q, const uint8_t *d_alive, int *found, u64 *sieve_sum,
                    u64 *per_point, double *ms)
{
    Workspace &w = g.ws;
    cudaStream_t st = g.stream;
    const u32 n = g.n, k = q.k;
    const u64 m = g.m;
    *found = 0;
    *sieve_sum = 0;

    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    TM_CUDA(cudaEventCreate(&ev0));
    TM_CUDA(cudaEventCreate(&ev1));
    TM_CUDA(cudaEventRecord(ev0, st));

    // slots: distinct colours of M ascending get consecutive slot ranges
    std::vector<u32> sb(g.num_colors, 0), sc(g.num_colors, 0);
    for (u32 c : q.multiset) sc[c]++;
    {
        u32 off = 0;
        for (u32 c = 0; c < g.num_colors; c++) { sb[c] = off; off += sc[c]; }
    }
    TM_TRY(w.slot_begin.reserve(g.num_colors * sizeof(u32)));
    TM_TRY(w.slot_count.reserve(g.num_colors * sizeof(u32)));
    TM_TRY(w.counters.reserve(64));
    if (w.host_pinned_bytes < 64 + LANES_MAX * 8) {
        if (w.host_pinned) cudaFreeHost(w.host_pinned);
        w.host_pinned = nullptr;
        TM_CUDA(cudaMallocHost(&w.host_pinned, 64 + LANES_MAX * 8));
        w.host_pinned_bytes = 64 + LANES_MAX * 8;
    }
    u32 *h_cnt = (u32 *)w.host_pinned;
    u64 *h_out = (u64 *)((char *)w.host_pinned + 64);
    TM_CUDA(cudaMemcpyAsync(w.slot_begin.p, sb.data(), g.num_colors * 4, cudaMemcpyHostToDevice, st));
    TM_CUDA(cudaMemcpyAsync(w.slot_count.p, sc.data(), g.num_colors * 4, cudaMemcpyHostToDevice, st));
    u32 *d_cnt = w.counters.as<u32>();

    // ---- prep: filter arcs (Sec. 7.1 (i)) ----
    cudaEvent_t pa = nullptr;
    TM_TRY(g.prof.begin(st, &pa));
    TM_TRY(w.vflag.reserve(std::max<u64>(n, 1)));
    TM_TRY(w.keep.reserve((m + 1) * 4));
    k_vflag<<<grid_for(n, 256), 256, 0, st>>>(n, g.d_color, w.slot_count.as<u32>(), d_alive, w.vflag.as<uint8_t>());
    k_keep<<<grid_for(m + 1, 256), 256, 0, st>>>(m, g.d_src, g.d_dst, g.d_time, w.vflag.as<uint8_t>(), q.t_min,
                                                 q.t_max, w.keep.as<u32>());
    g.prof.stats.launches += 2;
    TM_CUDA(cudaGetLastError());
    TM_TRY(exclusive_scan(g, w.keep.as<u32>(), m + 1, d_cnt + 0));
    TM_CUDA(cudaMemcpyAsync(h_cnt, d_cnt, 4, cudaMemcpyDeviceToHost, st));
    TM_CUDA(cudaStreamSynchronize(st));
    const u64 mf = h_cnt[0];

    u64 npts = q.p_end - q.p_begin;
    std::vector<u64> vals(npts, 0);
    if (mf > 0) {
        TM_TRY(w.f_src.reserve(mf * 4));
        TM_TRY(w.f_dst.reserve(mf * 4));
        TM_TRY(w.f_time.reserve(mf * 4));
        TM_TRY(w.pos.reserve(mf * 4));
        TM_TRY(w.mark.reserve((mf + 1) * 4));
        TM_TRY(w.cp_in.reserve(mf * 4));
        TM_TRY(w.cp_out.reserve(mf * 4));
        TM_TRY(w.seg_lo.reserve((u64)n * 4));
        TM_TRY(w.seg_hi.reserve((u64)n * 4));
        k_compact<<<grid_for(m, 256), 256, 0, st>>>(m, g.d_src, g.d_dst, g.d_time, w.keep.as<u32>(),
                                                    w.f_src.as<u32>(), w.f_dst.as<u32>(), w.f_time.as<u32>());
        TM_CUDA(cudaMemsetAsync(w.seg_lo.p, 0, (u64)n * 4, st));
        TM_CUDA(cudaMemsetAsync(w.seg_hi.p, 0, (u64)n * 4, st));
        TM_CUDA(cudaMemsetAsync(w.mark.p, 0, (mf + 1) * 4, st));
        k_segments<<<grid_for(mf, 256), 256, 0, st>>>(mf, w.f_dst.as<u32>(), w.seg_lo.as<u32>(), w.seg_hi.as<u32>());
        k_pos<<<grid_for(mf, 256), 256, 0, st>>>(mf, w.f_src.as<u32>(), w.f_time.as<u32>(), w.seg_lo.as<u32>(),
                                                 w.seg_hi.as<u32>(), w.pos.as<u32>(), w.mark.as<u32>());
        g.prof.stats.launches += 3;
        TM_CUDA(cudaGetLastError());
        TM_TRY(exclusive_scan(g, w.mark.as<u32>(), mf + 1, d_cnt + 1));
        k_checkpoints<<<grid_for(mf, 256), 256, 0, st>>>(mf, w.pos.as<u32>(), w.mark.as<u32>(), w.cp_in.as<u32>(),
                                                         w.cp_out.as<u32>());
        g.prof.stats.launches++;
        TM_CUDA(cudaGetLastError());
        TM_CUDA(cudaMemcpyAsync(h_cnt + 1, d_cnt + 1, 4, cudaMemcpyDeviceToHost, st));
    }
    TM_TRY(g.prof.end(st, pa, FAM_PREP));
    TM_CUDA(cudaStreamSynchronize(st));
    const u64 ncp = mf > 0 ? h_cnt[1] : 0;

    if (mf > 0) {
        // lane width: power of two >= 4, at most LANES_MAX
        u32 L = 4;
        while (L < LANES_MAX && L < npts) L <<= 1;
        const int T = (int)(L / 2 > 32 ? 32 : L / 2);
        const u32 lane_groups = L / (2 * T);
        TM_TRY(w.x.reserve((u64)n * L * 8));
        TM_TRY(w.C0.reserve(std::max<u64>(ncp, 1) * L * 8));
        TM_TRY(w.C1.reserve(std::max<u64>(ncp, 1) * L * 8));
        TM_TRY(w.out.reserve(L * 8));
        TM_TRY(w.wtab.reserve((u64)k * L * 8));
        const u32 chunk = 128;
        const u64 n_chunks = (mf + chunk - 1) / chunk;
        for (u32 r = 0; r < q.repeats; r++) {
            const QueryKeys keys = make_keys(mix64(q.seed + (u64)(r + 1) * TM_GOLDEN));
            u64 qsum = 0;
            for (u64 p0 = q.p_begin; p0 < q.p_end; p0 += L) {
                const u64 cnt = std::min<u64>(L, q.p_end - p0);
                cudaEvent_t ca = nullptr;
                TM_TRY(g.prof.begin(st, &ca));
                k_wtab<<<grid_for((u64)k * L, 128), 128, 0, st>>>(k, L, p0, keys, w.wtab.as<u64>());
                k_coef<<<grid_for((u64)n * L, 256), 256, 0, st>>>(n, L, w.vflag.as<uint8_t>(), g.d_color,
                                                                  w.slot_begin.as<u32>(), w.slot_count.as<u32>(),
                                                                  keys, w.wtab.as<u64>(), w.x.as<u64>());
                g.prof.stats.launches += 2;
                TM_CUDA(cudaGetLastError());
                TM_CUDA(cudaMemsetAsync(w.out.p, 0, L * 8, st));
                TM_TRY(g.prof.end(st, ca, FAM_COEF));
                LayerParams lp;
                lp.src = w.f_src.as<u32>();
                lp.dst = w.f_dst.as<u32>();
                lp.time = w.f_time.as<u32>();
                lp.cp_in = w.cp_in.as<u32>();
                lp.cp_out = w.cp_out.as<u32>();
                lp.seg_hi = w.seg_hi.as<u32>();
                lp.x = w.x.as<u64>();
                lp.out = w.out.as<u64>();
                lp.m_f = mf;
                lp.n_chunks = n_chunks;
                lp.ky = keys.ky;
                lp.L = L;
                lp.lane_groups = lane_groups;
                lp.chunk = chunk;
                lp.k = k;
                lp.start = q.start;
                lp.end = q.end;
                u64 *bufs[2] = {w.C0.as<u64>(), w.C1.as<u64>()};
                for (u32 ell = 2; ell <= k; ell++) {
                    lp.ell = ell;
                    lp.Cin = bufs[ell & 1];
                    lp.Cout = bufs[(ell + 1) & 1];
                    cudaEvent_t la = nullptr;
                    TM_TRY(g.prof.begin(st, &la));
                    TM_TRY(launch_layer(g, lp, T, n_chunks * lane_groups));
                    TM_TRY(g.prof.end(st, la, FAM_LAYER));
                }
                g.prof.stats.layer_arc_lanes += mf * (k - 1) * L;
                g.prof.stats.layer_cp_lanes += ncp * (k - 2) * L;
                // algorithmic bytes: per arc-lane one 8-byte read of the source
                // state (x at layer 2, a checkpoint above); per checkpoint-lane
                // one 8-byte write (layers 2..k-1)
                g.prof.stats.layer_bytes += (mf * (k - 1) + ncp * (k - 2)) * (u64)L * 8;
                g.prof.stats.layer_gf_muls += (mf * (k - 1) + ncp * (k - 2)) * (u64)L;
                TM_CUDA(cudaMemcpyAsync(h_out, w.out.p, L * 8, cudaMemcpyDeviceToHost, st));
                TM_CUDA(cudaStreamSynchronize(st));
                for (u64 i = 0; i < cnt; i++) {
                    qsum ^= h_out[i];
                    if (r == 0) vals[p0 - q.p_begin + i] = h_out[i];
                }
            }
            if (r == 0) *sieve_sum = qsum;
            if (qsum != 0) *found = 1;
        }
    }
    TM_CUDA(cudaEventRecord(ev1, st));
    TM_CUDA(cudaEventSynchronize(ev1));
    float fms = 0;
    cudaEventElapsedTime(&fms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (ms) *ms = fms;
    if (per_point) std::memcpy(per_point, vals.data(), npts * sizeof(u64));
    TM_TRY(g.prof.collect());
    return Status();
}

}  // namespace tmo

namespace tmo {

__global__ void k_vflag_mask(u32 n, const uint8_t *alive, uint8_t *vflag)
{
    u64 u = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n) vflag[u] = alive[u] ? 1 : 0;
}

Status gather_arcs(Graph &g, const uint8_t *d_alive, u32 t_min, u32 t_max, std::vector<u32> *src,
                   std::vector<u32> *dst, std::vector<u32> *time)
{
    Workspace &w = g.ws;
    cudaStream_t st = g.stream;
    const u64 m = g.m;
    TM_TRY(w.vflag.reserve(std::max<u64>(g.n, 1)));
    TM_TRY(w.keep.reserve((m + 1) * 4));
    TM_TRY(w.counters.reserve(64));
    k_vflag_mask<<<grid_for(g.n, 256), 256, 0, st>>>(g.n, d_alive, w.vflag.as<uint8_t>());
    k_keep<<<grid_for(m + 1, 256), 256, 0, st>>>(m, g.d_src, g.d_dst, g.d_time, w.vflag.as<uint8_t>(), t_min,
                                                 t_max, w.keep.as<u32>());
    g.prof.stats.launches += 2;
    TM_CUDA(cudaGetLastError());
    u32 *d_cnt = w.counters.as<u32>();
    TM_TRY(exclusive_scan(g, w.keep.as<u32>(), m + 1, d_cnt));
    u32 mf = 0;
    TM_CUDA(cudaMemcpyAsync(&mf, d_cnt, 4, cudaMemcpyDeviceToHost, st));
    TM_CUDA(cudaStreamSynchronize(st));
    src->assign(mf, 0);
    dst->assign(mf, 0);
    time->assign(mf, 0);
    if (mf == 0) return Status();
    TM_TRY(w.f_src.reserve((u64)mf * 4));
    TM_TRY(w.f_dst.reserve((u64)mf * 4));
    TM_TRY(w.f_time.reserve((u64)mf * 4));
    k_compact<<<grid_for(m, 256), 256, 0, st>>>(m, g.d_src, g.d_dst, g.d_time, w.keep.as<u32>(), w.f_src.as<u32>(),
                                                w.f_dst.as<u32>(), w.f_time.as<u32>());
    g.prof.stats.launches++;
    TM_CUDA(cudaGetLastError());
    TM_CUDA(cudaMemcpyAsync(src->data(), w.f_src.p, (u64)mf * 4, cudaMemcpyDeviceToHost, st));
    TM_CUDA(cudaMemcpyAsync(dst->data(), w.f_dst.p, (u64)mf * 4, cudaMemcpyDeviceToHost, st));
    TM_CUDA(cudaMemcpyAsync(time->data(), w.f_time.p, (u64)mf * 4, cudaMemcpyDeviceToHost, st));
    TM_CUDA(cudaStreamSynchronize(st));
    return Status();
}

}  // namespace tmo
