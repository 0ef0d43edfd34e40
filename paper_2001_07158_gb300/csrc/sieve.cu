// sieve.cu -- per-query kernels of the constrained multilinear sieve.
//
// For one query the device runs, per lane batch of L sieve points:
//   1. prep (once per query): keep the arcs whose endpoints carry a query
//      colour and whose time is in the window (Sec. 8.1 preprocessing (i):
//      vertices whose colour is not in M contribute x_u = 0), compact them in
//      (dst, time, src) order, find for every arc e = (a -> b, t) the last
//      in-arc of a with time < t ("pos"), and number the distinct pos values
//      ("checkpoints": the only prefix values any later arc reads);
//   2. coefficients x_u^A = sum_{d in S_c(u)} v_{u,d} W_d^A (Lemma 6.5,
//      eq. motif:1) for every lane;
//   3. layers l = 2..k of eq. (gen-polynomial:3), edge-centric: for arc e into
//      b, H_l[e] = y_{e,l-1} * P_{a,l-1,t(e)-1}; P_{b,l,i} is x_b times the XOR
//      of H_l over b's in-arcs with time <= i (the "+ P_{u,l,i-1}" stay term
//      is the running prefix); it is stored only at checkpoints; the last
//      layer XORs x_b * (sum of H_k over b's in-arcs) into the lane's sum.
// P_{a,1,i} = x_a for all i (the base case, read at i = 0 as well), so layer 2
// reads x directly.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <tuple>

#include "gf64.cuh"
#include "internal.h"
#include "layer.cuh"
#include "scan.cuh"

namespace tmo {

// The device status word (TM_STATUS_* bits; see status_word): kernels of this
// file name it directly, kernels elsewhere get its address in their params.
static __device__ u32 g_status_word;

// ---------------------------------------------------------------------------
// Per-query preparation
// ---------------------------------------------------------------------------
// vflag[u] = 1 for vertices with a query colour (and alive); act[u] the same
// as u32 flags (n+1 entries, act[n] = 0) for the active-vertex scan.
__global__ void k_vflag(u32 n, const u32 *color, const u32 *slot_count, const uint8_t *alive, uint8_t *vflag,
                        u32 *act)
{
    u64 u = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (u > n) return;
    if (u == n) { act[n] = 0; return; }
    bool f = slot_count[color[u]] > 0;
    if (alive) f = f && alive[u];
    vflag[u] = f ? 1 : 0;
    act[u] = f ? 1u : 0u;
}

// act[] holds exclusive offsets: list[act[u]] = u for active u.
__global__ void k_active_list(u32 n, const u32 *act, u32 *list)
{
    u64 u = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n && act[u + 1] != act[u]) list[act[u]] = (u32)u;
}

// ---------------------------------------------------------------------------
// Arc filter (Sec. 8.1 (i)).  Arc e is kept iff both endpoints are flagged,
// its time lies in the window and, for EC-PathMotif (Sec. 7.3), its time is
// one of the tuple's.  Two passes over tiles of 4096 arcs in arc order:
//   k_filter_count writes one bit per arc (word j of the mask covers arcs
//     32j..32j+31) and the tile's kept count;
//   after an exclusive scan of the tile counts, k_filter_compact writes the
//     kept arcs, in arc order, from the mask alone.
// The destination's flag is tested first: arcs are sorted by destination,
// so those reads are nearly sequential, and the scattered source flag and the
// time are read only for arcs that pass the tests before them.
// Where few arcs have a flagged destination, the first pass goes by vertex
// instead (k_filter_count_v): one warp per flagged destination walks its
// in-segment (the graph's in-segment offsets) and writes the same mask bits
// and tile counts, so the arcs of unflagged destinations are never read.
// ---------------------------------------------------------------------------
namespace {

const int FILTER_THREADS = 256;
const int FILTER_ROUNDS = 16;                                  // arcs per thread
const int FILTER_TILE = FILTER_THREADS * FILTER_ROUNDS;        // 4096 arcs
const int FILTER_WORDS = FILTER_TILE / 32;                     // 128 mask words

// Time window and EC tuple of the filter (true for an untimed filter).
__device__ __forceinline__ bool filter_time_ok(const ArcFilter &f, u32 t)
{
    bool in = t >= f.t_min && (f.t_max == 0 || t <= f.t_max);
    if (in && f.n_times) {
        // constant indices keep the tuple in the parameter space
        bool hit = false;
#pragma unroll
        for (int r = 0; r < TMOTIF_KMAX; r++) hit |= (r < (int)f.n_times) && f.times[r] == t;
        in = hit;
    }
    return in;
}

__global__ void __launch_bounds__(FILTER_THREADS)
k_filter_count(u64 m, const u32 *src, const u32 *dst, const u32 *time, const uint8_t *vflag, ArcFilter f, u32 *bits,
               u32 *tile_count)
{
    __shared__ u32 warp_count[FILTER_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const u64 base = (u64)blockIdx.x * FILTER_TILE;
    const bool timed = f.t_min != 0 || f.t_max != 0 || f.n_times != 0;
    u32 d[FILTER_ROUNDS];
    bool k[FILTER_ROUNDS];
#pragma unroll
    for (int i = 0; i < FILTER_ROUNDS; i++) {
        const u64 e = base + (u64)i * FILTER_THREADS + threadIdx.x;
        d[i] = e < m ? dst[e] : 0u;
    }
#pragma unroll
    for (int i = 0; i < FILTER_ROUNDS; i++) {
        const u64 e = base + (u64)i * FILTER_THREADS + threadIdx.x;
        k[i] = e < m && vflag[d[i]];
    }
#pragma unroll
    for (int i = 0; i < FILTER_ROUNDS; i++) {
        const u64 e = base + (u64)i * FILTER_THREADS + threadIdx.x;
        if (k[i]) d[i] = src[e];  // d[] now holds the source
    }
#pragma unroll
    for (int i = 0; i < FILTER_ROUNDS; i++)
        if (k[i]) k[i] = vflag[d[i]];
    if (timed) {
#pragma unroll
        for (int i = 0; i < FILTER_ROUNDS; i++) {
            if (!k[i]) continue;
            k[i] = filter_time_ok(f, time[base + (u64)i * FILTER_THREADS + threadIdx.x]);
        }
    }
    u32 count = 0;
#pragma unroll
    for (int i = 0; i < FILTER_ROUNDS; i++) {
        const u32 b = __ballot_sync(0xffffffffu, k[i]);
        if (lane == 0) bits[(u64)blockIdx.x * FILTER_WORDS + i * (FILTER_THREADS / 32) + w] = b;
        count += __popc(b);
    }
    if (lane == 0) warp_count[w] = count;
    __syncthreads();
    if (threadIdx.x == 0) {
        u32 t = 0;
        for (int i = 0; i < FILTER_THREADS / 32; i++) t += warp_count[i];
        tile_count[blockIdx.x] = t;
    }
}

// First pass by vertex: resident warps take the flagged destinations v of
// list[0, *n_list) (ascending) and walk each in-segment [in_off[v],
// in_off[v + 1]) in rounds of 32 arcs, testing the source's flag and the time.
// A round's kept bits land in at most two mask words, ORed in (a word can
// hold the arcs of two destinations), and its count goes to the tiles of
// those words.  The mask and the tile counts are zero before the launch.
__global__ void __launch_bounds__(FILTER_THREADS)
k_filter_count_v(const u32 *list, const u32 *n_list, const u32 *in_off, const u32 *src, const u32 *time,
                 const uint8_t *vflag, ArcFilter f, u32 n, u64 m, u32 *bits, u32 *tile_count)
{
    const int lane = threadIdx.x & 31;
    const bool timed = f.t_min != 0 || f.t_max != 0 || f.n_times != 0;
    const u64 nl = *n_list;
    const u64 warps = (u64)gridDim.x * (FILTER_THREADS / 32);
    for (u64 i = (u64)blockIdx.x * (FILTER_THREADS / 32) + (threadIdx.x >> 5); i < nl; i += warps) {
        const u32 v = list[i];  // uniform in the warp
        if (!TM_IN(v, n, &g_status_word)) continue;
        const u64 lo = in_off[v], hi = in_off[v + 1];
        if (!TM_IN(hi, m + 1, &g_status_word) || !TM_IN(lo, hi + 1, &g_status_word)) continue;
        for (u64 b = lo; b < hi; b += 32) {
            const u64 e = b + lane;
            bool ok = false;
            if (e < hi) {
                const u32 a = src[e];
                ok = TM_IN(a, n, &g_status_word) && vflag[a];
                if (ok && timed) ok = filter_time_ok(f, time[e]);
            }
            const u32 mask = __ballot_sync(0xffffffffu, ok);
            if (lane == 0 && mask) {
                const u64 w0 = b >> 5;
                const u32 sh = (u32)(b & 31);
                const u32 lo_bits = mask << sh, hi_bits = sh ? mask >> (32 - sh) : 0u;
                if (lo_bits) {
                    atomicOr(&bits[w0], lo_bits);
                    atomicAdd(&tile_count[w0 / FILTER_WORDS], (u32)__popc(lo_bits));
                }
                if (hi_bits) {
                    atomicOr(&bits[w0 + 1], hi_bits);
                    atomicAdd(&tile_count[(w0 + 1) / FILTER_WORDS], (u32)__popc(hi_bits));
                }
            }
        }
    }
}

// tile_off: exclusive offsets of the tiles' kept counts.  One warp per tile,
// in 4 rounds of 32 mask words (1024 arcs): lane l owns word l of the round;
// a warp scan of the words' counts places each word's kept arcs, whose tile
// indices the lane lists in shared memory in arc order; the warp then copies
// the listed arcs with independent loads and contiguous stores.
__global__ void __launch_bounds__(FILTER_THREADS)
k_filter_compact(const u32 *__restrict__ src, const u32 *__restrict__ dst, const u32 *__restrict__ time,
                 const u32 *__restrict__ bits, const u32 *__restrict__ tile_off, u32 ntiles, u32 *__restrict__ f_src,
                 u32 *__restrict__ f_dst, u32 *__restrict__ f_time)
{
    __shared__ uint16_t list[FILTER_THREADS / 32][1024];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const u64 tile = (u64)blockIdx.x * (FILTER_THREADS / 32) + w;
    if (tile >= ntiles) return;
    uint16_t *q = list[w];
    const u64 abase = tile * FILTER_TILE;
    u32 out = tile_off[tile];
    for (int r = 0; r < FILTER_WORDS / 32; r++) {
        const int wi = 32 * r + lane;  // word index in the tile
        u32 b = bits[tile * FILTER_WORDS + wi];
        const u32 c = __popc(b);
        u32 incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u32 y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const u32 total = __shfl_sync(0xffffffffu, incl, 31);
        if (total == 0) continue;
        u32 p = incl - c;
        while (b) {
            const int bit = __ffs(b) - 1;
            b &= b - 1;
            q[p++] = (uint16_t)(wi * 32 + bit);
        }
        __syncwarp();
        for (u32 i = lane; i < total; i += 32) {
            const u64 e = abase + q[i];
            f_src[out + i] = src[e];
            f_dst[out + i] = dst[e];
            f_time[out + i] = time[e];
        }
        __syncwarp();
        out += total;
    }
}

}  // namespace

// First pass of the arc filter: the keep mask in w.kbits, the tile offsets in
// w.ftiles and the kept count to d_total (device u32).  With a vertex list
// (the flagged destinations, ascending, their count at d_nlist) and in_off,
// by vertex; otherwise by tiles of arcs.
Status filter_arcs_count(cudaStream_t st, Workspace &w, const u32 *src, const u32 *dst, const u32 *time,
                         const u32 *in_off, u32 n, u64 m, const uint8_t *vflag, const ArcFilter &f, u32 *d_total,
                         u64 *launches, const u32 *vlist, const u32 *d_nlist)
{
    const u64 ntiles = std::max<u64>(1, (m + FILTER_TILE - 1) / FILTER_TILE);
    TM_TRY(w.kbits.reserve(ntiles * FILTER_WORDS * 4));
    TM_TRY(w.ftiles.reserve(ntiles * 4));
    if (vlist && d_nlist && in_off) {
        TM_CUDA(cudaMemsetAsync(w.kbits.p, 0, ntiles * FILTER_WORDS * 4, st));
        TM_CUDA(cudaMemsetAsync(w.ftiles.p, 0, ntiles * 4, st));
        const u64 blocks = std::max<u64>(1, std::min<u64>((n + 7) / 8, (u64)8 * sm_count()));
        k_filter_count_v<<<(unsigned)blocks, FILTER_THREADS, 0, st>>>(vlist, d_nlist, in_off, src, time, vflag, f, n,
                                                                      m, w.kbits.as<u32>(), w.ftiles.as<u32>());
    } else {
        k_filter_count<<<(unsigned)ntiles, FILTER_THREADS, 0, st>>>(m, src, dst, time, vflag, f, w.kbits.as<u32>(),
                                                                    w.ftiles.as<u32>());
    }
    if (launches) *launches += 1;
    TM_CUDA(cudaGetLastError());
    return exclusive_scan_on(st, w.block_sums, w.ftiles.as<u32>(), ntiles, d_total, launches);
}

// Second pass: the kept arcs, in arc order, into (o_src, o_dst, o_time).
Status filter_arcs_compact(cudaStream_t st, Workspace &w, const u32 *src, const u32 *dst, const u32 *time, u64 m,
                           u32 *o_src, u32 *o_dst, u32 *o_time, u64 *launches)
{
    const u64 ntiles = std::max<u64>(1, (m + FILTER_TILE - 1) / FILTER_TILE);
    const u64 per_block = FILTER_THREADS / 32;
    k_filter_compact<<<(unsigned)((ntiles + per_block - 1) / per_block), FILTER_THREADS, 0, st>>>(
        src, dst, time, w.kbits.as<u32>(), w.ftiles.as<u32>(), (u32)ntiles, o_src, o_dst, o_time);
    if (launches) *launches += 1;
    TM_CUDA(cudaGetLastError());
    return Status();
}

// len[d] += (end - start) of d's in-segment: the segment's first arc subtracts
// its index and its last arc adds its index + 1 (two atomics per segment).
__global__ void k_in_len(u64 m, const u32 *dst, u32 n, u32 *len)
{
    const u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    const u32 d = dst[e];
    if (!TM_IN(d, n, &g_status_word)) return;
    if (e == 0 || dst[e - 1] != d) atomicSub(&len[d], (u32)e);
    if (e + 1 == m || dst[e + 1] != d) atomicAdd(&len[d], (u32)(e + 1));
}

Status build_in_off(Graph &g, cudaStream_t st, DevBuf &tiles, u32 *d_total)
{
    g.d_in_off = nullptr;
    if (g.m >= 0xFFFFFFFFull) return Status();  // u32 offsets: the filter reads destinations instead
    const u64 bytes = ((u64)g.n + 1) * 4;
    TM_TRY(dev_alloc((void **)&g.d_in_off, bytes, st));
    TM_CUDA(cudaMemsetAsync(g.d_in_off, 0, bytes, st));
    if (g.m) k_in_len<<<(unsigned)((g.m + 255) / 256), 256, 0, st>>>(g.m, g.d_dst, g.n, g.d_in_off);
    TM_CUDA(cudaGetLastError());
    TM_TRY(exclusive_scan_on(st, tiles, g.d_in_off, (u64)g.n + 1, d_total, nullptr));
    g.resident_bytes += bytes;
    return Status();
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
__global__ void k_segments(u64 mf, const u32 *f_dst, u32 *seg_lo, u32 *seg_hi, u32 n)
{
    u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= mf) return;
    u32 d = f_dst[e];
    if (!TM_IN(d, n, &g_status_word)) return;
    if (e == 0 || f_dst[e - 1] != d) seg_lo[d] = (u32)e;
    if (e + 1 == mf || f_dst[e + 1] != d) seg_hi[d] = (u32)(e + 1);
}

// pos[e] = last in-arc of src(e) with time < time(e) (strictly increasing times,
// Sec. 4), or NONE; marks that arc as a checkpoint.
__global__ void k_pos(u64 mf, const u32 *f_src, const u32 *f_time, const u32 *seg_lo, const u32 *seg_hi,
                      u32 *pos, u32 *mark, u32 n)
{
    u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= mf) return;
    u32 a = f_src[e], t = f_time[e];
    if (!TM_IN(a, n, &g_status_word)) return;
    u32 lo = seg_lo[a], hi = seg_hi[a];
    if (!TM_IN(hi, mf + 1, &g_status_word) || !TM_IN(lo, (u64)hi + 1, &g_status_word)) return;
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

// mark[] holds exclusive checkpoint numbers (length mf+1).  With rec (the
// staged layer form), also each arc's record {dst, cp_in, cp_out, src}; with
// max_seg, the longest in-segment (from its first arc and seg_hi).
__global__ void k_checkpoints(u64 mf, const u32 *pos, const u32 *ck, u32 *cp_in, u32 *cp_out, const u32 *f_src,
                              const u32 *f_dst, uint4 *rec, const u32 *seg_hi, u32 *max_seg)
{
    u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= mf) return;
    if (max_seg) {  // one atomic per warp, on the warp's longest segment
        const u32 len = (e == 0 || f_dst[e - 1] != f_dst[e]) ? seg_hi[f_dst[e]] - (u32)e : 0u;
        const unsigned act = __activemask();
        const u32 wmax = __reduce_max_sync(act, len);
        if (wmax && (threadIdx.x & 31) == (u32)(__ffs(act) - 1)) atomicMax(max_seg, wmax);
    }
    u32 p = pos[e];
    if (p != NONE && !TM_IN(p, mf, &g_status_word)) return;
    const u32 ci = (p == NONE) ? NONE : ck[p];
    u32 c = ck[e];
    const u32 co = (ck[e + 1] != c) ? c : NONE;
    cp_in[e] = ci;
    cp_out[e] = co;
    if (rec) rec[e] = make_uint4(f_dst[e], ci, co, f_src[e]);
}

// ---------------------------------------------------------------------------
// Chunk order of single-job layer launches: a chunk is heavy when its arc
// range, extended to whole in-segments as the layer team extends it, holds
// more than twice the chunk size (a long in-segment starts in it).  Teams take
// heavy chunks first, so that a long segment never starts last and keeps one
// team busy after the others have run out of work.
// ---------------------------------------------------------------------------
__global__ void k_chunk_heavy(u64 mf, u64 n_chunks, u32 chunk, const u32 *dst, const u32 *seg_hi, u32 *flag)
{
    const u64 c = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (c > n_chunks) return;
    if (c == n_chunks) { flag[c] = 0; return; }
    const u64 b0 = c * chunk, b1 = min(b0 + chunk, mf);
    u64 begin = b0, stop = b1;
    if (b0 > 0 && dst[b0] == dst[b0 - 1]) begin = seg_hi[dst[b0]];
    if (b1 < mf && dst[b1] == dst[b1 - 1]) stop = seg_hi[dst[b1]];
    flag[c] = (stop > begin && stop - begin > 2ull * chunk) ? 1u : 0u;
}

// off[] holds the exclusive offsets of the heavy flags (n_chunks + 1 entries,
// off[n_chunks] = number of heavy chunks): heavy chunks first, then the others,
// each group in index order.
__global__ void k_chunk_order(u64 n_chunks, const u32 *off, u32 *order)
{
    const u64 c = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_chunks) return;
    const u32 o = off[c];
    const bool heavy = off[c + 1] != o;
    order[heavy ? o : off[n_chunks] + (u32)(c - o)] = (u32)c;
}

// ---------------------------------------------------------------------------
// Coefficients (Lemma 6.5, eq. motif:1)
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

// x_u^A = sum_{d in S_c(u)} v_{u,d} W_d^A for the active vertices: one warp
// per vertex; v_{u,d} is common to all lanes, so the warp builds its nibble
// table once per slot and each lane's product is 16 table loads.
__global__ void __launch_bounds__(256) k_coef(u32 n_act, const u32 *list, u32 L, const u32 *color,
                                              const u32 *slot_begin, const u32 *slot_count, QueryKeys keys,
                                              const u64 *wtab, u64 *x, u32 n, u32 num_colors, u32 k)
{
    __shared__ __align__(2048) u64 tabs[8][256];  // tables on 2 KB boundaries
    u64 *tab = tabs[threadIdx.x >> 5];
    const int tt = threadIdx.x & 31;
    const u64 v = (u64)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (v >= n_act) return;  // whole warp leaves together
    const u32 u = list[v];
    if (!TM_IN(u, n, &g_status_word)) return;
    const u32 c = color[u];
    if (!TM_IN(c, num_colors, &g_status_word)) return;
    const u32 d0 = slot_begin[c], d1 = d0 + slot_count[c];
    if (!TM_IN(d1, k + 1, &g_status_word)) return;
    u64 s[4] = {0, 0, 0, 0};  // lanes tt, tt + 32, tt + 64, tt + 96 (L <= 128)
    for (u32 d = d0; d < d1; d++) {
        __syncwarp();
        gf_table_build(tab, coef_v(keys, u, d), tt, 32);
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 4; i++)
            if ((u32)tt + 32 * i < L) s[i] ^= gf_table_mul(tab, wtab[(u64)d * L + tt + 32 * i]);
    }
#pragma unroll
    for (int i = 0; i < 4; i++)
        if ((u32)tt + 32 * i < L) x[(u64)u * L + tt + 32 * i] = s[i];
}

// Coefficients by multiplier table (large lists): x_u^A = sum_d v_{u,d} W_d^A
// read the other way round.  W_d^A is common to every vertex of slot d, so a
// block holds the nibble tables of W_d^A for all k slots and a group of LG
// lanes (k * LG tables of 2 KB, built once per block) and each thread takes a
// vertex: per slot of its colour one v_{u,d}, then LG lane products of 16
// table loads.  The vertices come grouped by colour (slist), so the threads
// of a warp read the same table at each step.

// Grouping the active vertices by colour: gcnt[slot_begin[c]] counts colour c
// (k counters; one atomic per colour per warp), then every vertex takes a
// place in its colour's range of slist.
__global__ void k_group_count(u32 n_act, const u32 *list, const u32 *color, const u32 *slot_begin, u32 *gcnt)
{
    const u64 v = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n_act) return;
    const u32 g = slot_begin[color[list[v]]];
    const unsigned act = __activemask();
    const unsigned same = __match_any_sync(act, g);
    if ((threadIdx.x & 31) == (u32)(__ffs(same) - 1)) atomicAdd(&gcnt[g], (u32)__popc(same));
}

// gcnt[0..k): counts, gcnt[k..2k): cursors (zero); slist gets each colour's
// vertices in the range that the counts' exclusive prefix gives.
__global__ void k_group_scatter(u32 n_act, const u32 *list, const u32 *color, const u32 *slot_begin, u32 k,
                                u32 *gcnt, u32 *slist)
{
    const u64 v = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n_act) return;
    const u32 u = list[v];
    const u32 g = slot_begin[color[u]];
    if (!TM_IN(g, k, &g_status_word)) return;
    u32 base = 0;
    for (u32 i = 0; i < g; i++) base += gcnt[i];
    const unsigned act = __activemask();
    const unsigned same = __match_any_sync(act, g);
    const int lead = __ffs(same) - 1;
    u32 first = 0;
    if ((int)(threadIdx.x & 31) == lead) first = atomicAdd(&gcnt[k + g], (u32)__popc(same));
    first = __shfl_sync(same, first, lead);
    const u32 rank = __popc(same & ((1u << (threadIdx.x & 31)) - 1u));
    slist[base + first + rank] = u;
}

const int COEF_T_THREADS = 512;
const u64 COEF_T_SMEM = 192 * 1024;  // tables; plus 2 KB for the alignment

// Lanes per block of k_coef_t: the largest power of two <= L whose k tables
// per lane fit COEF_T_SMEM, at least 4 (k <= TMOTIF_KMAX).
static u32 coef_t_lanes(u32 k, u32 L)
{
    u32 lg = std::min<u32>(L, 16);
    while (lg > 4 && (u64)k * lg * 2048 > COEF_T_SMEM) lg >>= 1;
    return lg;
}

template <int LG>
__global__ void __launch_bounds__(COEF_T_THREADS) k_coef_t(u32 n_act, const u32 *slist, u32 L, u32 k,
                                                           const u32 *color, const u32 *slot_begin,
                                                           const u32 *slot_count, QueryKeys keys, const u64 *wtab,
                                                           u64 *x, u32 n, u32 num_colors, u32 groups)
{
    extern __shared__ __align__(16) u64 smem[];
    const u32 sa = (u32)__cvta_generic_to_shared(smem);
    u64 *tabs = smem + (((2048u - (sa & 2047u)) & 2047u) >> 3);  // 2 KB boundary
    const u32 group = blockIdx.x % groups, a0 = group * LG;
    const u32 warp = threadIdx.x >> 5, tt = threadIdx.x & 31, nwarps = COEF_T_THREADS / 32;
    // table (d, a) at tabs + (d * LG + a) * 256: nibble table of W_d^{a0 + a}
    for (u32 t = warp; t < k * LG; t += nwarps)
        gf_table_build(tabs + (u64)t * 256, wtab[(u64)(t / LG) * L + a0 + t % LG], tt, 32);
    __syncthreads();
    const u64 step = (u64)(gridDim.x / groups) * COEF_T_THREADS;
    for (u64 i = (u64)(blockIdx.x / groups) * COEF_T_THREADS + threadIdx.x; i < n_act; i += step) {
        const u32 u = slist[i];
        if (!TM_IN(u, n, &g_status_word)) continue;
        const u32 c = color[u];
        if (!TM_IN(c, num_colors, &g_status_word)) continue;
        const u32 d0 = slot_begin[c], d1 = d0 + slot_count[c];
        if (!TM_IN(d1, k + 1, &g_status_word)) continue;
        u64 acc[LG];
#pragma unroll
        for (int a = 0; a < LG; a++) acc[a] = 0;
        for (u32 d = d0; d < d1; d++) {
            const u64 v = coef_v(keys, u, d);
            const u64 *td = tabs + (u64)d * LG * 256;
#pragma unroll
            for (int a = 0; a < LG; a++) acc[a] ^= gf_table_mul(td + a * 256, v);
        }
        ulonglong2 *out = (ulonglong2 *)(x + (u64)u * L + a0);
#pragma unroll
        for (int a = 0; a < LG; a += 2) out[a / 2] = make_ulonglong2(acc[a], acc[a + 1]);
    }
}

// ---------------------------------------------------------------------------
// Layer kernel: eq. (gen-polynomial:3), one walk length per job per launch.
// MULTI = false: the single job in `one` (read from parameter space);
// MULTI = true: the team's job is found in the prefix of team counts.
template <int T, bool TAB, bool MULTI, int LPT, bool INNER>
__device__ __forceinline__ void layer_kernel(const LayerParams &one, const LayerParams *__restrict__ jobs,
                                             const u64 *__restrict__ team_prefix, u32 njobs)
{
    extern __shared__ __align__(16) u64 smem[];
    // team tables of 2 KB each, starting on a 2 KB boundary of shared memory
    // (the launch adds 2 KB of slack for the rounding)
    const u32 sa = (u32)__cvta_generic_to_shared(smem);
    u64 *tab = smem + (((2048u - (sa & 2047u)) & 2047u) >> 3) + (size_t)(threadIdx.x / T) * 256;
    const u64 team = (u64)blockIdx.x * (blockDim.x / T) + threadIdx.x / T;
    // one team per team slot ...
    const u64 total = MULTI ? team_prefix[njobs] : one.n_chunks * one.lane_groups;
    auto run = [&](u64 t) {
        if (!MULTI) {
            layer_team<T, TAB, LPT, false, INNER>(one, t, tab);
            return;
        }
        u32 lo = 0, hi = njobs;  // last job with team_prefix[job] <= t
        while (hi - lo > 1) {
            const u32 mid = (lo + hi) >> 1;
            if (team_prefix[mid] <= t) lo = mid;
            else hi = mid;
        }
        layer_team<T, TAB, LPT, false>(jobs[lo], t - team_prefix[lo], tab);
    };
    if (!one.queue) {
        if (team < total) run(team);
        return;
    }
    // ... or resident teams take team indices in order from the counter until
    // none is left, so chunks of uneven work (long in-segments, small and
    // large jobs) leave no tail of idle SMs
    const u32 team_mask = (T == 32) ? 0xffffffffu : (((1u << T) - 1u) << (((threadIdx.x & 31) / T) * T));
    for (;;) {
        unsigned long long t = 0;
        if (threadIdx.x % T == 0) t = atomicAdd(one.queue, 1ull);
        t = __shfl_sync(team_mask, t, 0, T);
        if (t >= total) return;
        run(t);
    }
}

// k_layer: the compiler's own register budget for 256-thread blocks;
// k_layer_mb: the blocks of 256 threads per SM the allocation must allow
// (2: up to 128 registers per thread, 4: 64).  These are the register shapes
// the autotuner picks from.  INNER (single job, 2 < l < k): the form without
// the first and last layers' cases.
template <int T, bool TAB, bool MULTI, int LPT, bool INNER = false>
__global__ void __launch_bounds__(256) k_layer(LayerParams one, const LayerParams *__restrict__ jobs,
                                               const u64 *__restrict__ team_prefix, u32 njobs)
{
    layer_kernel<T, TAB, MULTI, LPT, INNER>(one, jobs, team_prefix, njobs);
}

template <int T, bool TAB, int LPT, int MINB, bool INNER = false>
__global__ void __launch_bounds__(256, MINB) k_layer_mb(LayerParams one)
{
    layer_kernel<T, TAB, false, LPT, INNER>(one, nullptr, nullptr, 0);
}

// The staged form (variant 4 of the warp-team classes L = 32, 64, 128;
// single-job launches with a team counter): the same team body with each
// team's arc metadata staged in shared memory by bulk copies.  Dynamic shared
// memory: the eight teams' staging areas, then their tables on 2 KB
// boundaries (STAGED_SMEM bytes).
constexpr size_t STAGED_SMEM = 8 * sizeof(TeamStage) + 8 * 2048 + 2048;

template <int LPT, bool INNER>
__global__ void __launch_bounds__(256) k_layer_staged(LayerParams one)
{
    extern __shared__ __align__(16) u64 smem[];
    TeamStage *ts = (TeamStage *)smem + threadIdx.x / 32;
    u64 *after = (u64 *)((TeamStage *)smem + 8);
    const u32 sa = smem_u32(after);
    u64 *tab = after + (((2048u - (sa & 2047u)) & 2047u) >> 3) + (size_t)(threadIdx.x / 32) * 256;
    if (threadIdx.x % 32 == 0) stage_init(ts);
    __syncwarp();
    StageState ss;
    const u64 total = one.n_chunks * one.lane_groups;
    for (;;) {
        unsigned long long t = 0;
        if (threadIdx.x % 32 == 0) t = atomicAdd(one.queue, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= total) break;
        layer_team<32, true, LPT, false, INNER, true>(one, t, tab, ts, &ss);
    }
    // a team whose wait ran out may still have copies in flight into its
    // buffers: wait for them (each wait bounded) before the block's shared
    // memory is released
    if (ss.broken)
        for (int b = 0; b < 2; b++)
            if (ss.pending & (1u << b)) stage_wait(ts, b, (ss.phase >> b) & 1u);
}

// out[lane] ^= XOR over chunks of partial[chunk * L + lane] (L a power of two
// <= 256).  A block of 256 threads reads 256 / L whole chunk rows per round
// (thread t: lane t % L of row t / L), rows strided over the grid; the block
// folds its rows in shared memory and adds one atomic per lane.
const int REDUCE_THREADS = 256;
__global__ void __launch_bounds__(REDUCE_THREADS) k_reduce_partials(const u64 *partial, u64 n_chunks, u32 L, u64 *out)
{
    __shared__ u64 red[REDUCE_THREADS];
    const u32 t = threadIdx.x, rows = REDUCE_THREADS / L;
    const u64 step = (u64)gridDim.x * rows;
    u64 s = 0;
#pragma unroll 4
    for (u64 c = (u64)blockIdx.x * rows + t / L; c < n_chunks; c += step) s ^= partial[c * L + t % L];
    red[t] = s;
    __syncthreads();
    for (u32 r = rows / 2; r > 0; r >>= 1) {
        if (t < r * L) red[t] ^= red[t + r * L];
        __syncthreads();
    }
    if (t < L && red[t]) atomicXor(&out[t], red[t]);
}

// ---------------------------------------------------------------------------
// Diagnostic multiply kernel
// ---------------------------------------------------------------------------
__global__ void k_gf_mul(const u64 *a, const u64 *b, u64 *out, u64 n)
{
    u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = gf_mul(a[i], b[i]);
}

// Throughput probe of the two product forms on register-resident data: every
// warp runs `iters` rounds; a round multiplies 64 lanes (2 per thread) by one
// multiplier, which changes every round.  method 0: register multiply;
// method 1: shared-memory nibble table built by the warp, then looked up for
// 64 lanes (2 per thread); method 2: the same table for 128 lanes (4 per
// thread).
template <int METHOD>
__global__ void __launch_bounds__(256) k_gf_probe(u32 iters, u64 seed, u64 *sink)
{
    __shared__ __align__(2048) u64 tabs[8][256];  // tables on 2 KB boundaries
    u64 *tab = tabs[threadIdx.x >> 5];
    const int tt = threadIdx.x & 31;
    constexpr int LPT = METHOD == 2 ? 4 : 2;  // lanes per thread
    u64 a[LPT], acc[LPT];
    a[0] = mix64(seed + blockIdx.x * 256 + threadIdx.x);
#pragma unroll
    for (int i = 1; i < LPT; i++) a[i] = mix64(a[i - 1]);
#pragma unroll
    for (int i = 0; i < LPT; i++) acc[i] = 0;
    u64 y = mix64(seed ^ blockIdx.x);
    for (u32 it = 0; it < iters; it++) {
        if (METHOD == 0) {
#pragma unroll
            for (int i = 0; i < LPT; i++) acc[i] ^= gf_mul(y, a[i]);
        } else {
            __syncwarp();
            gf_table_build(tab, y, tt, 32);
            __syncwarp();
#pragma unroll
            for (int i = 0; i < LPT; i++) acc[i] ^= gf_table_mul(tab, a[i]);
        }
#pragma unroll
        for (int i = 0; i < LPT; i++) a[i] += acc[(i + 1) % LPT];
        y += TM_GOLDEN;
    }
    u64 r = 0;
#pragma unroll
    for (int i = 0; i < LPT; i++) r ^= acc[i];
    if (r == 0x5151ull) sink[0] = r;
}

Status gf_probe(int method, u32 iters, double *ms, u64 *products)
{
    u64 *sink = nullptr;
    TM_CUDA(cudaMalloc(&sink, 64));
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned blocks = (unsigned)sms * 8;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    for (int pass = 0; pass < 2; pass++) {  // warm-up launch, then the timed one
        if (pass == 1) cudaEventRecord(a);
        const u32 n = pass ? iters : 4;
        if (method == 0) k_gf_probe<0><<<blocks, 256>>>(n, 1 + 6 * pass, sink);
        else if (method == 1) k_gf_probe<1><<<blocks, 256>>>(n, 1 + 6 * pass, sink);
        else k_gf_probe<2><<<blocks, 256>>>(n, 1 + 6 * pass, sink);
    }
    cudaEventRecord(b);
    cudaError_t e = cudaEventSynchronize(b);
    float f = 0;
    cudaEventElapsedTime(&f, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    if (e != cudaSuccess) return cuda_fail(e, "gf_probe");
    TM_CUDA(cudaGetLastError());
    *ms = f;
    *products = (u64)blocks * 256 * (method == 2 ? 4 : 2) * iters;
    return Status();
}

// ---------------------------------------------------------------------------
// Device status word
// ---------------------------------------------------------------------------
static std::mutex g_status_mu;
static u32 *g_status_ptr[256];  // device address of g_status_word, per device

Status status_word(u32 **p)
{
    int dev = 0;
    TM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return fail(TMOTIF_ERR_UNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lock(g_status_mu);
    if (!g_status_ptr[dev]) {
        void *a = nullptr;
        TM_CUDA(cudaGetSymbolAddress(&a, g_status_word));
        g_status_ptr[dev] = (u32 *)a;
    }
    *p = g_status_ptr[dev];
    return Status();
}

__global__ void k_status_take(u32 *word, u32 *out) { *out = atomicExch(word, 0u); }

Status status_take_enqueue(cudaStream_t st, u32 *d_slot, u32 *h_slot)
{
    u32 *word = nullptr;
    TM_TRY(status_word(&word));
    k_status_take<<<1, 1, 0, st>>>(word, d_slot);
    TM_CUDA(cudaGetLastError());
    TM_CUDA(cudaMemcpyAsync(h_slot, d_slot, 4, cudaMemcpyDeviceToHost, st));
    return Status();
}

Status status_result(u32 taken)
{
    if (taken & TM_STATUS_STAGE_TIMEOUT)
        return fail(TMOTIF_ERR_TIMEOUT, "a staged layer launch's bulk copy did not complete within its wait limit");
    if (taken & TM_STATUS_BOUNDS)
        return fail(TMOTIF_ERR_INVALID, "a device bounds check failed (the access was skipped; results are invalid)");
    if (taken) return fail(TMOTIF_ERR_CUDA, "unknown device status bits");
    return Status();
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
// Host orchestration: jobs.
// ---------------------------------------------------------------------------
static inline unsigned grid_for(u64 items, int threads) { return (unsigned)((items + threads - 1) / threads); }

static const u32 LANES_MAX = 128;  // lanes per batch (one warp owns up to 128 lanes)
static const u32 CHUNK = 128;     // arcs per team chunk (whole in-segments), untuned
static const u32 CHUNK_MIN = 64;  // smallest chunk the autotuner tries (partials sized for it)
static const size_t PIN_BYTES = 64 + LANES_MAX * 8;

static Status ensure_pinned(Workspace &w, size_t bytes = PIN_BYTES)
{
    if (w.host_pinned_bytes >= bytes) return Status();
    if (w.host_pinned) cudaFreeHost(w.host_pinned);
    w.host_pinned = nullptr;
    w.host_pinned_bytes = 0;
    TM_CUDA(cudaMallocHost(&w.host_pinned, bytes));
    w.host_pinned_bytes = bytes;
    return Status();
}

// Team width, lane groups and chunk count of a job's layer launches from its
// lane width and shape: 2 lanes per thread (T = L / 2, at most 32), 4 at
// L = 128; variant 1 at L = 128 splits the lanes over two 64-lane teams of
// the 2-lanes-per-thread form (one table build per team).
static void set_team_shape(Job &j)
{
    j.T = j.L / 2 > 32 ? 32 : j.L / 2;
    j.lane_groups = (j.L == 128 && j.variant == 1) ? 2 : 1;
    j.n_chunks = (j.mf + j.chunk - 1) / j.chunk;
}

size_t job_bytes(const Job &j)
{
    const u64 n = j.g->n, m = j.mf ? j.mf : j.g->m, L = j.L ? j.L : LANES_MAX;
    const u64 ncp = j.mf ? j.ncp : m;
    return (size_t)(n * (1 + 12) + j.g->m / 8 + 4096 + m * 28 + n * L * 8 + 2 * ncp * L * 8 +
                    ((m + CHUNK_MIN - 1) / CHUNK_MIN) * L * 8 + 4096);
}

// Lane width of a job: a power of two >= 4, at most LANES_MAX, halved while
// the lane-proportional buffers (x, two checkpoint buffers of ncp rows, chunk
// partials) would not fit the device memory left.  Per-point values do not
// depend on the lane width.
static Status lane_width(const Job &j, u64 ncp, u32 *out)
{
    const Workspace &w = *j.ws;
    const u64 npts = j.q.p_end - j.q.p_begin;
    u32 L = 4;
    while (L < LANES_MAX && L < npts) L <<= 1;
    size_t room = 0;
    TM_TRY(device_headroom(&room));
    room += w.x.bytes + w.C0.bytes + w.C1.bytes + w.partial.bytes;
    const u64 per_lane = ((u64)j.g->n + 2 * std::max<u64>(ncp, 1) + (j.mf + CHUNK_MIN - 1) / CHUNK_MIN) * 8;
    while (L > 4 && per_lane * L > room / 10 * 9) L >>= 1;
    *out = L;
    return Status();
}

// Lists of at least COEF_T_MIN_LANES vertex-lanes at lane widths up to
// COEF_T_MAX_L take the coefficients by multiplier table (k_coef_t); the
// others one warp per vertex (k_coef), whose per-vertex table is then shared
// by 64 or 128 lanes and which was faster there.
static const u64 COEF_T_MIN_LANES = 1ull << 20;
static const u32 COEF_T_MAX_L = 32;

template <int LG>
static Status launch_coef_t(cudaStream_t s, u32 blocks, u32 groups, size_t smem, u32 n_act, const u32 *slist, u32 L,
                            u32 k, const Graph &g, const Workspace &w, const QueryKeys &keys)
{
    static bool attr_set[64] = {false};
    int dev = 0;
    TM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(TMOTIF_ERR_CUDA, "device index");
    if (!attr_set[dev]) {
        TM_CUDA(cudaFuncSetAttribute(k_coef_t<LG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(COEF_T_SMEM + 2048)));
        attr_set[dev] = true;
    }
    k_coef_t<LG><<<blocks, COEF_T_THREADS, smem, s>>>(n_act, slist, L, k, g.d_color, w.slot_begin.as<u32>(),
                                                       w.slot_count.as<u32>(), keys, w.wtab.as<u64>(),
                                                       w.x.as<u64>(), g.n, g.num_colors, groups);
    return Status();
}

// Coefficients x_u^A and W_d^A of the lane batch at p0 for repeat r, lane
// width L, on stream s (2 launches; the first batch of a query by table also
// groups the active vertices by colour, 2 launches).
static Status launch_coef(Job &j, cudaStream_t s, u32 L, u64 p0, u32 r)
{
    Graph &g = *j.g;
    Workspace &w = *j.ws;
    const u32 k = j.q.k;
    const QueryKeys keys = make_keys(mix64(j.q.seed + (u64)(r + j.rep_offset + 1) * TM_GOLDEN));
    cudaEvent_t ca = nullptr;
    TM_TRY(j.prof->begin(s, &ca));
    k_wtab<<<grid_for((u64)k * L, 128), 128, 0, s>>>(k, L, p0, keys, w.wtab.as<u64>());
    j.prof->stats.launches += 1;
    if (j.n_act && L <= COEF_T_MAX_L && j.n_act * L >= COEF_T_MIN_LANES) {
        if (!j.slist_ready) {
            TM_TRY(w.slist.reserve(j.n_act * 4));
            TM_TRY(w.gcount.reserve(2 * (u64)TMOTIF_KMAX * 4));
            TM_CUDA(cudaMemsetAsync(w.gcount.p, 0, 2 * (u64)k * 4, s));
            k_group_count<<<grid_for(j.n_act, 256), 256, 0, s>>>((u32)j.n_act, w.act_list.as<u32>(), g.d_color,
                                                                  w.slot_begin.as<u32>(), w.gcount.as<u32>());
            k_group_scatter<<<grid_for(j.n_act, 256), 256, 0, s>>>((u32)j.n_act, w.act_list.as<u32>(), g.d_color,
                                                                    w.slot_begin.as<u32>(), k, w.gcount.as<u32>(),
                                                                    w.slist.as<u32>());
            j.prof->stats.launches += 2;
            TM_CUDA(cudaGetLastError());
            j.slist_ready = true;
        }
        const u32 lg = coef_t_lanes(k, L), groups = L / lg;
        const u32 blocks = groups * std::max<u32>(1, (u32)sm_count() / groups);
        const size_t smem = (size_t)k * lg * 2048 + 2048;
        const u32 *sl = w.slist.as<u32>();
        if (lg == 16) TM_TRY(launch_coef_t<16>(s, blocks, groups, smem, (u32)j.n_act, sl, L, k, g, w, keys));
        else if (lg == 8) TM_TRY(launch_coef_t<8>(s, blocks, groups, smem, (u32)j.n_act, sl, L, k, g, w, keys));
        else TM_TRY(launch_coef_t<4>(s, blocks, groups, smem, (u32)j.n_act, sl, L, k, g, w, keys));
        j.prof->stats.launches += 1;
    } else if (j.n_act) {
        k_coef<<<(unsigned)((j.n_act + 7) / 8), 256, 0, s>>>((u32)j.n_act, w.act_list.as<u32>(), L, g.d_color,
                                                              w.slot_begin.as<u32>(), w.slot_count.as<u32>(), keys,
                                                              w.wtab.as<u64>(), w.x.as<u64>(), g.n, g.num_colors, k);
        j.prof->stats.launches += 1;
    }
    TM_CUDA(cudaGetLastError());
    return j.prof->end(s, ca, FAM_COEF);
}

// Arcs whose destination's colour is in the multiset (before masks and the
// time window), from the graph's colour-pair counts; m where there are none.
static u64 flagged_dst_arcs(const Graph &g, const QuerySpec &q)
{
    if (g.pair_hist.empty()) return g.m;
    std::vector<bool> in(g.num_colors, false);
    for (u32 c : q.multiset) in[c] = true;
    u64 s = 0;
    for (u32 a = 0; a < g.num_colors; a++)
        for (u32 b = 0; b < g.num_colors; b++)
            if (in[b]) s += g.pair_hist[(size_t)a * g.num_colors + b];
    return s;
}

Status job_prep(Job &j)
{
    Graph &g = *j.g;
    Workspace &w = *j.ws;
    const cudaStream_t st = j.st;
    const QuerySpec &q = j.q;
    const u32 n = g.n;
    const u64 m = g.m;
    u64 *launches = (u64 *)&j.prof->stats.launches;

    // slots: distinct colours of M ascending get consecutive slot ranges
    std::vector<u32> sb(g.num_colors, 0), sc(g.num_colors, 0);
    for (u32 c : q.multiset) sc[c]++;
    for (u32 c = 0, off = 0; c < g.num_colors; c++) { sb[c] = off; off += sc[c]; }
    TM_TRY(w.slot_begin.reserve(g.num_colors * sizeof(u32)));
    TM_TRY(w.slot_count.reserve(g.num_colors * sizeof(u32)));
    TM_TRY(w.counters.reserve(64));
    TM_TRY(ensure_pinned(w));
    u32 *h_cnt = (u32 *)w.host_pinned;
    TM_CUDA(cudaMemcpyAsync(w.slot_begin.p, sb.data(), g.num_colors * 4, cudaMemcpyHostToDevice, st));
    TM_CUDA(cudaMemcpyAsync(w.slot_count.p, sc.data(), g.num_colors * 4, cudaMemcpyHostToDevice, st));
    u32 *d_cnt = w.counters.as<u32>();

    w.order_chunk = 0;  // the chunk order belongs to the previous query's arcs
    j.slist_ready = false;  // the active vertices grouped by colour, for this query
    // filter arcs (Sec. 8.1 (i): colours outside M, masked vertices, window)
    cudaEvent_t pa = nullptr;
    TM_TRY(j.prof->begin(st, &pa));
    TM_TRY(w.vflag.reserve(std::max<u64>(n, 1)));
    TM_TRY(w.act.reserve(((u64)n + 1) * 4));
    TM_TRY(w.act_list.reserve(std::max<u64>(n, 1) * 4));
    k_vflag<<<grid_for((u64)n + 1, 256), 256, 0, st>>>(n, g.d_color, w.slot_count.as<u32>(), j.d_alive,
                                                       w.vflag.as<uint8_t>(), w.act.as<u32>());
    *launches += 1;
    TM_CUDA(cudaGetLastError());
    TM_TRY(exclusive_scan_on(st, w.block_sums, w.act.as<u32>(), (u64)n + 1, d_cnt + 2, launches));
    k_active_list<<<grid_for(n, 256), 256, 0, st>>>(n, w.act.as<u32>(), w.act_list.as<u32>());
    *launches += 1;
    // the filter by flagged destination (the active list) where such arcs are
    // a small share of all
    const bool by_vertex = g.d_in_off && flagged_dst_arcs(g, q) * 10 < (u64)m * 3;
    TM_TRY(filter_arcs_count(st, w, g.d_src, g.d_dst, g.d_time, g.d_in_off, g.n, m, w.vflag.as<uint8_t>(), q.filter(),
                             d_cnt + 0, launches, by_vertex ? w.act_list.as<u32>() : nullptr, d_cnt + 2));
    TM_CUDA(cudaMemcpyAsync(h_cnt, d_cnt, 12, cudaMemcpyDeviceToHost, st));
    TM_CUDA(cudaStreamSynchronize(st));
    j.mf = h_cnt[0];
    j.n_act = h_cnt[2];
    j.ncp = 0;
    if (j.mf > 0) {
        const u64 mf = j.mf;
        TM_TRY(w.f_src.reserve(mf * 4));
        TM_TRY(w.f_dst.reserve(mf * 4));
        TM_TRY(w.f_time.reserve((mf + 4) * 4));  // the staged form copies times in 16-byte units
        TM_TRY(w.rec.reserve(mf * 16));
        TM_TRY(w.pos.reserve(mf * 4));
        TM_TRY(w.mark.reserve((mf + 1) * 4));
        TM_TRY(w.cp_in.reserve(mf * 4));
        TM_TRY(w.cp_out.reserve(mf * 4));
        TM_TRY(w.seg_lo.reserve((u64)n * 4));
        TM_TRY(w.seg_hi.reserve((u64)n * 4));
        TM_TRY(filter_arcs_compact(st, w, g.d_src, g.d_dst, g.d_time, m, w.f_src.as<u32>(), w.f_dst.as<u32>(),
                                   w.f_time.as<u32>(), launches));
        TM_CUDA(cudaMemsetAsync(w.seg_lo.p, 0, (u64)n * 4, st));
        TM_CUDA(cudaMemsetAsync(w.seg_hi.p, 0, (u64)n * 4, st));
        TM_CUDA(cudaMemsetAsync(w.mark.p, 0, (mf + 1) * 4, st));
        TM_CUDA(cudaMemsetAsync(d_cnt + 14, 0, 4, st));
        k_segments<<<grid_for(mf, 256), 256, 0, st>>>(mf, w.f_dst.as<u32>(), w.seg_lo.as<u32>(), w.seg_hi.as<u32>(),
                                                      n);
        k_pos<<<grid_for(mf, 256), 256, 0, st>>>(mf, w.f_src.as<u32>(), w.f_time.as<u32>(), w.seg_lo.as<u32>(),
                                                 w.seg_hi.as<u32>(), w.pos.as<u32>(), w.mark.as<u32>(), n);
        *launches += 2;
        TM_CUDA(cudaGetLastError());
        TM_TRY(exclusive_scan_on(st, w.block_sums, w.mark.as<u32>(), mf + 1, d_cnt + 1, launches));
        k_checkpoints<<<grid_for(mf, 256), 256, 0, st>>>(mf, w.pos.as<u32>(), w.mark.as<u32>(), w.cp_in.as<u32>(),
                                                         w.cp_out.as<u32>(), w.f_src.as<u32>(), w.f_dst.as<u32>(),
                                                         w.rec.as<uint4>(), w.seg_hi.as<u32>(), d_cnt + 14);
        *launches += 1;
        TM_CUDA(cudaGetLastError());
        TM_CUDA(cudaMemcpyAsync(h_cnt + 1, d_cnt + 1, 4, cudaMemcpyDeviceToHost, st));
        TM_CUDA(cudaMemcpyAsync(h_cnt + 14, d_cnt + 14, 4, cudaMemcpyDeviceToHost, st));
    }
    TM_TRY(j.prof->end(st, pa, FAM_PREP));
    TM_CUDA(cudaStreamSynchronize(st));
    j.max_seg = 0;
    if (j.mf > 0) {
        j.ncp = h_cnt[1];
        j.max_seg = h_cnt[14];
    }

    const u64 npts = q.p_end - q.p_begin;
    j.vals.assign(npts, 0);
    j.r = 0;
    j.p0 = q.p_begin;
    j.qsum = 0;
    j.found = 0;
    j.sieve_sum = 0;
    j.done = (j.mf == 0);
    if (j.done) return Status();
    u32 L = 0;
    TM_TRY(lane_width(j, j.ncp, &L));
    j.L = L;
    j.chunk = CHUNK;
    j.variant = 0;
    {  // the launch shape pinned or tuned for this graph and lane width, else
       // one tuned on this device for a layer of about the same size
        std::lock_guard<std::mutex> lock(layer_tune_mutex());
        auto it = g.layer_tune.find(L);
        std::pair<u32, u32> shape;
        if (it != g.layer_tune.end()) {
            j.chunk = it->second.first;
            j.variant = it->second.second;
        } else if (tuned_shape(L, j.mf, &shape)) {
            g.layer_tune[L] = shape;
            j.chunk = shape.first;
            j.variant = shape.second;
        }
    }
    set_team_shape(j);
    TM_TRY(w.x.reserve((u64)n * L * 8));
    TM_TRY(w.C0.reserve(std::max<u64>(j.ncp, 1) * L * 8));
    TM_TRY(w.C1.reserve(std::max<u64>(j.ncp, 1) * L * 8));
    TM_TRY(w.out.reserve(L * 8));
    TM_TRY(w.wtab.reserve((u64)q.k * L * 8));
    TM_TRY(w.partial.reserve(((j.mf + CHUNK_MIN - 1) / CHUNK_MIN) * L * 8));
    TM_TRY(w.queue.reserve(sizeof(unsigned long long)));
    if (j.localize) {
        TM_TRY(w.arc_sum.reserve(j.mf * 8));
        TM_CUDA(cudaMemsetAsync(w.arc_sum.p, 0, j.mf * 8, st));
    }
    return Status();
}

Status job_batch_begin(Job &j)
{
    Workspace &w = *j.ws;
    const cudaStream_t st = j.st;
    const u32 L = j.L;
    j.ky = make_keys(mix64(j.q.seed + (u64)(j.r + j.rep_offset + 1) * TM_GOLDEN)).ky;
    TM_TRY(launch_coef(j, st, L, j.p0, j.r));
    TM_CUDA(cudaMemsetAsync(w.out.p, 0, L * 8, st));
    j.ell = 2;
    return Status();
}

LayerParams job_layer_params(const Job &j)
{
    const Workspace &w = *j.ws;
    LayerParams lp;
    lp.src = w.f_src.as<u32>();
    lp.dst = w.f_dst.as<u32>();
    lp.time = w.f_time.as<u32>();
    lp.cp_in = w.cp_in.as<u32>();
    lp.cp_out = w.cp_out.as<u32>();
    lp.seg_hi = w.seg_hi.as<u32>();
    lp.x = w.x.as<u64>();
    u64 *bufs[2] = {w.C0.as<u64>(), w.C1.as<u64>()};
    lp.Cin = bufs[j.ell & 1];
    lp.Cout = bufs[(j.ell + 1) & 1];
    lp.partial = w.partial.as<u64>();
    lp.arc_sum = j.localize ? w.arc_sum.as<u64>() : nullptr;
    lp.m_f = j.mf;
    lp.n_chunks = j.n_chunks;
    lp.ky = j.ky;
    lp.L = j.L;
    lp.lane_groups = j.lane_groups;
    lp.chunk = j.chunk;
    lp.ell = j.ell;
    lp.k = j.q.k;
    lp.start = j.q.start;
    lp.end = j.q.end;
    lp.T = j.T;
    lp.queue = w.queue.as<unsigned long long>();
    lp.rec = w.rec.as<uint4>();
    lp.n_vert = j.g->n;
    lp.n_cp = j.ncp;
    lp.order = (w.order_chunk == j.chunk && w.order_chunk != 0) ? w.order.as<u32>() : nullptr;
    u32 *status = nullptr;
    if (status_word(&status).ok()) lp.status = status;
    return lp;
}

// One launch of the layer kernel.  MINB = 0: k_layer (single- or multi-job);
// MINB > 0: k_layer_mb with that register bound (single-job only).
template <int T, bool TAB, int LPT, int MINB, bool INNER>
static Status launch_layer_f(cudaStream_t st, const LayerParams &one, const LayerParams *jobs,
                             const u64 *prefix, u32 njobs, u64 teams)
{
    const int threads = 256;
    const u64 teams_per_block = threads / T;
    const unsigned blocks = (unsigned)((teams + teams_per_block - 1) / teams_per_block);
    const size_t smem = TAB ? teams_per_block * 256 * 8 + 2048 : 16;
    if (smem > 48 * 1024) {  // above the default limit: opt in (per call, so per device and thread-safe)
        if constexpr (MINB == 0) {
            TM_CUDA(cudaFuncSetAttribute(njobs == 0 ? k_layer<T, TAB, false, LPT, INNER> : k_layer<T, TAB, true, LPT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        } else {
            TM_CUDA(cudaFuncSetAttribute(k_layer_mb<T, TAB, LPT, MINB, INNER>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        }
    }
    if (!blocks) return Status();
    unsigned grid = blocks;
    if (one.queue) {  // resident blocks only, fed from the team counter
        auto resident = [&](const void *kernel) {
            int nb = 0;
            const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem);
            return (e == cudaSuccess && nb > 0) ? nb : 1;
        };
        int per_sm = 1;
        if constexpr (MINB == 0) {
            static const int single = resident((const void *)k_layer<T, TAB, false, LPT, INNER>);
            static const int multi = resident((const void *)k_layer<T, TAB, true, LPT>);
            per_sm = njobs == 0 ? single : multi;
        } else {
            static const int mb = resident((const void *)k_layer_mb<T, TAB, LPT, MINB, INNER>);
            per_sm = mb;
        }
        grid = (unsigned)std::min<u64>(blocks, (u64)per_sm * sm_count());
        TM_CUDA(cudaMemsetAsync(one.queue, 0, sizeof(unsigned long long), st));
    }
    if constexpr (MINB == 0) {
        if (njobs == 0) k_layer<T, TAB, false, LPT, INNER><<<grid, threads, smem, st>>>(one, jobs, prefix, njobs);
        else k_layer<T, TAB, true, LPT><<<grid, threads, smem, st>>>(one, jobs, prefix, njobs);
    } else {
        if (njobs != 0) return fail(TMOTIF_ERR_UNSUPPORTED, "multi-job launches use the default kernel form");
        k_layer_mb<T, TAB, LPT, MINB, INNER><<<grid, threads, smem, st>>>(one);
    }
    return Status();
}

static std::atomic<u32> g_stage_extra_tx{0};

Status debug_stage_timeout(bool on)
{
#ifdef TMOTIF_CHECKED
    g_stage_extra_tx.store(on ? 16u : 0u);
    return Status();
#else
    (void)on;
    return fail(TMOTIF_ERR_UNSUPPORTED, "the forced staged-copy timeout exists only in the checked build");
#endif
}

// One launch of the staged form (single job, warp teams of LPT lanes per
// thread): resident blocks only, fed from the team counter.
template <int LPT, bool INNER>
static Status launch_staged_f(cudaStream_t st, const LayerParams &one, u64 teams)
{
    if (!one.queue || !one.rec) return fail(TMOTIF_ERR_UNSUPPORTED, "the staged layer form needs a job workspace");
    // bulk copies start on 16-byte boundaries: the arrays' bases must be aligned
    if (((uintptr_t)one.rec | (uintptr_t)one.time) & 15u)
        return fail(TMOTIF_ERR_UNSUPPORTED, "the staged layer form needs 16-byte aligned arc arrays");
    const int threads = 256;
    const u64 blocks = (teams + 7) / 8;
    if (!blocks) return Status();
    static const int per_sm = [] {
        int nb = 0;
        const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_layer_staged<LPT, INNER>, 256,
                                                                            STAGED_SMEM);
        return (e == cudaSuccess && nb > 0) ? nb : 1;
    }();
    const unsigned grid = (unsigned)std::min<u64>(blocks, (u64)per_sm * sm_count());
    TM_CUDA(cudaMemsetAsync(one.queue, 0, sizeof(unsigned long long), st));
    LayerParams p = one;
    p.stage_extra_tx = g_stage_extra_tx.load();
    k_layer_staged<LPT, INNER><<<grid, threads, STAGED_SMEM, st>>>(p);
    return Status();
}

template <int LPT>
static Status launch_staged(cudaStream_t st, const LayerParams &one, u64 teams)
{
    if (one.ell > 2 && one.ell < one.k) return launch_staged_f<LPT, true>(st, one, teams);
    return launch_staged_f<LPT, false>(st, one, teams);
}

// Single-job launches of inner layers (2 < l < k) take the INNER form.
template <int T, bool TAB, int LPT, int MINB>
static Status launch_layer_t(cudaStream_t st, const LayerParams &one, const LayerParams *jobs,
                             const u64 *prefix, u32 njobs, u64 teams)
{
    if (njobs == 0 && one.ell > 2 && one.ell < one.k)
        return launch_layer_f<T, TAB, LPT, MINB, true>(st, one, jobs, prefix, njobs, teams);
    return launch_layer_f<T, TAB, LPT, MINB, false>(st, one, jobs, prefix, njobs, teams);
}

// One kernel form per lane width L (the launch class): L = T * LPT.  The
// register shape is the variant of the table forms at 2 lanes per thread:
// 0 = the compiler's budget, 1 = 4 blocks per SM, 2 = 2.  At L = 32 the
// default team is a whole warp at one lane per thread, which keeps the warp
// convergent (two 16-thread teams would walk different arcs); variant 3 is
// the 16-thread team at 2 lanes per thread.  Other forms and multi-job
// launches have only variant 0.
template <int T, bool TAB, int LPT>
static Status launch_layer_v(cudaStream_t st, u32 variant, const LayerParams &one, const LayerParams *jobs,
                             const u64 *prefix, u32 njobs, u64 teams)
{
    if constexpr (TAB && LPT == 2 && T != 16) {  // T = 16 only as the L = 32 variant 3
        if (njobs == 0 && variant == 1) return launch_layer_t<T, TAB, LPT, 4>(st, one, jobs, prefix, njobs, teams);
        if (njobs == 0 && variant == 2) return launch_layer_t<T, TAB, LPT, 2>(st, one, jobs, prefix, njobs, teams);
    }
    return launch_layer_t<T, TAB, LPT, 0>(st, one, jobs, prefix, njobs, teams);
}

static Status launch_layer_class(cudaStream_t st, u32 L, u32 variant, const LayerParams &one,
                                 const LayerParams *jobs, const u64 *prefix, u32 njobs, u64 teams)
{
    if (variant == 4 && njobs == 0) {  // the staged form of the warp-team classes
        if (L == 32) return launch_staged<1>(st, one, teams);
        if (L == 64) return launch_staged<2>(st, one, teams);
        if (L == 128) return launch_staged<4>(st, one, teams);
    }
    switch (L) {
        case 4: return launch_layer_v<2, false, 2>(st, variant, one, jobs, prefix, njobs, teams);
        case 8: return launch_layer_v<4, false, 2>(st, variant, one, jobs, prefix, njobs, teams);
        case 16: return launch_layer_v<8, true, 2>(st, variant, one, jobs, prefix, njobs, teams);
        case 32:
            if (variant == 3 && njobs == 0) return launch_layer_t<16, true, 2, 0>(st, one, jobs, prefix, njobs, teams);
            return launch_layer_v<32, true, 1>(st, variant, one, jobs, prefix, njobs, teams);
        case 64: return launch_layer_v<32, true, 2>(st, variant, one, jobs, prefix, njobs, teams);
        default:
            if (variant == 1 && njobs == 0)  // two 64-lane teams per chunk (lane_groups = 2)
                return launch_layer_t<32, true, 2, 0>(st, one, jobs, prefix, njobs, teams);
            return launch_layer_v<32, true, 4>(st, variant, one, jobs, prefix, njobs, teams);
    }
}

static void count_layer(Profiler *prof, const Job &j, u32 lane_groups)
{
    const u64 L = j.L, k = j.q.k;
    prof->stats.layer_arc_lanes += j.mf * L;
    if (j.ell < k) prof->stats.layer_cp_lanes += j.ncp * L;
    // algorithmic bytes: per arc-lane one 8-byte read of the source state (x at
    // layer 2, a checkpoint above); per checkpoint-lane one 8-byte write
    const u64 writes = (j.ell < k) ? j.ncp : 0;
    prof->stats.layer_bytes += (j.mf + writes) * L * 8;
    prof->stats.layer_gf_muls += (j.mf + writes) * L;
    if (j.T >= 8) {
        prof->stats.layer_table_muls += j.mf * L;
        prof->stats.layer_table_builds += j.mf * lane_groups;
    }
}

// The heavy-first chunk order of a job's layer launches at its current chunk
// size, built once per (query, chunk size) for launches of at least
// ORDER_MIN_CHUNKS chunks whose longest in-segment exceeds twice the chunk
// (3 small launches on the job's stream); other launches keep index order.
static const u64 ORDER_MIN_CHUNKS = 1024;

static Status ensure_order(Job &j)
{
    Workspace &w = *j.ws;
    // no segment longer than twice the chunk: every chunk is light, and index
    // order is the order
    if (j.n_chunks < ORDER_MIN_CHUNKS || j.max_seg <= 2ull * j.chunk || w.order_chunk == j.chunk) return Status();
    const u64 nc = j.n_chunks;
    TM_TRY(w.order.reserve((2 * nc + 1) * 4));
    u32 *flag = w.order.as<u32>() + nc;  // nc + 1 flags, then offsets
    k_chunk_heavy<<<grid_for(nc + 1, 256), 256, 0, j.st>>>(j.mf, nc, j.chunk, w.f_dst.as<u32>(), w.seg_hi.as<u32>(),
                                                          flag);
    TM_CUDA(cudaGetLastError());
    TM_TRY(exclusive_scan_on(j.st, w.block_sums, flag, nc + 1, w.counters.as<u32>() + 13,
                             (u64 *)&j.prof->stats.launches));
    k_chunk_order<<<grid_for(nc, 256), 256, 0, j.st>>>(nc, flag, w.order.as<u32>());
    TM_CUDA(cudaGetLastError());
    j.prof->stats.launches += 2;
    w.order_chunk = j.chunk;
    return Status();
}

// One job's layer launch in its own (tuned or pinned) shape.
static Status launch_one(cudaStream_t st, Job &j, Profiler *prof)
{
    TM_TRY(ensure_order(j));
    cudaEvent_t la = nullptr;
    TM_TRY(prof->begin(st, &la));
    TM_TRY(launch_layer_class(st, j.L, j.variant, job_layer_params(j), nullptr, nullptr, 0,
                              j.n_chunks * j.lane_groups));
    TM_CUDA(cudaGetLastError());
    TM_TRY(prof->end(st, la, FAM_LAYER));
    prof->stats.launches++;
    prof->stats.layer_launches++;
    count_layer(prof, j, j.lane_groups);
    return Status();
}

Status launch_layers(cudaStream_t st, const std::vector<Job *> &jobs, DevBuf &dev_params, void *host_params,
                     size_t host_params_bytes, Profiler *prof)
{
    if (jobs.empty()) return Status();
    if (jobs.size() == 1) return launch_one(st, *jobs[0], prof);
    // group by lane width; per class: job table + team prefix.  A job alone
    // in its class keeps its own launch shape.
    const u32 classes[6] = {4, 8, 16, 32, 64, 128};
    size_t off = 0;
    for (u32 Lc : classes) {
        std::vector<Job *> cls;
        for (Job *j : jobs)
            if (j->L == Lc) cls.push_back(j);
        if (cls.empty()) continue;
        if (cls.size() == 1) {
            TM_TRY(launch_one(st, *cls[0], prof));
            continue;
        }
        // job table, team prefix, then the launch's team counter
        const size_t need = cls.size() * sizeof(LayerParams) + (cls.size() + 2) * sizeof(u64);
        const size_t at = (off + 255) & ~(size_t)255;
        if (at + need > host_params_bytes) return fail(TMOTIF_ERR_UNSUPPORTED, "too many jobs in one layer launch");
        LayerParams *hp = (LayerParams *)((char *)host_params + at);
        u64 *hpre = (u64 *)((char *)host_params + at + cls.size() * sizeof(LayerParams));
        u64 teams = 0;
        for (size_t i = 0; i < cls.size(); i++) {
            hp[i] = job_layer_params(*cls[i]);
            hp[i].lane_groups = 1;  // multi-job launches use the default form of each class
            hp[i].queue = nullptr;
            hpre[i] = teams;
            teams += cls[i]->n_chunks;
            count_layer(prof, *cls[i], 1);
        }
        hpre[cls.size()] = teams;
        TM_TRY(dev_params.reserve(host_params_bytes));
        char *dbase = (char *)dev_params.p + at;
        TM_CUDA(cudaMemcpyAsync(dbase, (char *)host_params + at, need, cudaMemcpyHostToDevice, st));
        LayerParams head = hp[0];
        head.queue = (unsigned long long *)(dbase + cls.size() * sizeof(LayerParams) + (cls.size() + 1) * sizeof(u64));
        cudaEvent_t la = nullptr;
        TM_TRY(prof->begin(st, &la));
        TM_TRY(launch_layer_class(st, Lc, 0, head, (const LayerParams *)dbase,
                                  (const u64 *)(dbase + cls.size() * sizeof(LayerParams)), (u32)cls.size(), teams));
        TM_CUDA(cudaGetLastError());
        TM_TRY(prof->end(st, la, FAM_LAYER));
        prof->stats.launches++;
        prof->stats.layer_launches++;
        off = at + need;
    }
    return Status();
}

// Shapes the autotuner found, per device, lane width and layer size class
// (floor(log2(arcs))), shared by every graph of the process.
static std::mutex g_tune_mu;

std::mutex &layer_tune_mutex()
{
    static std::mutex mu;
    return mu;
}
static std::map<std::tuple<int, u32, u32>, std::pair<u32, u32>> g_tuned;

static std::tuple<int, u32, u32> tune_key(u32 L, u64 mf)
{
    int dev = 0;
    cudaGetDevice(&dev);
    u32 b = 0;
    while ((mf >> (b + 1)) != 0) b++;
    return {dev, L, b};
}

std::string tuner_export()
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    std::string out;
    for (const auto &kv : g_tuned) {
        char line[96];
        std::snprintf(line, sizeof(line), "%d %u %u %u %u\n", std::get<0>(kv.first), std::get<1>(kv.first),
                      std::get<2>(kv.first), kv.second.first, kv.second.second);
        out += line;
    }
    return out;
}

Status tuner_import(const std::string &text)
{
    std::map<std::tuple<int, u32, u32>, std::pair<u32, u32>> add;
    size_t at = 0;
    while (at < text.size()) {
        size_t eol = text.find('\n', at);
        if (eol == std::string::npos) eol = text.size();
        const std::string line = text.substr(at, eol - at);
        at = eol + 1;
        if (line.find_first_not_of(" \t\r") == std::string::npos) continue;  // blank line
        int dev = -1;
        unsigned L = 0, b = 0, chunk = 0, variant = 0;
        char extra = 0;
        if (std::sscanf(line.c_str(), "%d %u %u %u %u %c", &dev, &L, &b, &chunk, &variant, &extra) != 5 || dev < 0 ||
            dev > 255 || b > 63 || !layer_shape_valid(L, chunk, variant))
            return fail(TMOTIF_ERR_INVALID, "bad tuner line: \"" + line + "\"");
        add[{dev, L, b}] = {chunk, variant};
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const auto &kv : add) g_tuned[kv.first] = kv.second;
    return Status();
}

bool tuned_shape(u32 L, u64 mf, std::pair<u32, u32> *shape)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tuned.find(tune_key(L, mf));
    if (it == g_tuned.end()) return false;
    *shape = it->second;
    return true;
}

// Autotuner of the layer kernel's launch shape.  On the first lane batch of
// a decision whose (graph, lane width) has no entry yet and whose layers
// hold at least 2^22 arc-lanes, layer 3 is launched
// for every candidate -- arcs per team chunk in {64, ..., 1024} x register
// shape {compiler's budget, 4 blocks per SM, 2 blocks per SM} (table forms at
// 2 lanes per thread, L = 16 and 64; at L = 32 the one-lane warp team and
// the two-lane 16-thread team; at L = 128 the four-lane warp team and two
// two-lane teams) -- twice, each
// launch timed by CUDA events on the job's stream.  The fastest shape (least
// of its two times) is kept for the graph and used by every later job on it
// with that lane width; the layer then runs once more in that shape, whose
// output (checkpoints, or at the last layer the per-chunk partial sums that
// the readout reduces) the rest of the decision uses.
static Status tune_layer(Job &j)
{
    struct Cand {
        u32 chunk, variant;
        float ms;
    };
    std::vector<Cand> cands;
    std::vector<u32> variants{0};
    if (j.L == 16) variants = {0, 1, 2};
    if (j.L == 32) variants = {0, 3, 4};
    if (j.L == 64) variants = {0, 1, 2, 4};
    if (j.L == 128) variants = {0, 1, 4};
    for (u32 c : {64u, 128u, 256u, 512u, 1024u})
        for (u32 v : variants) cands.push_back({c, v, 1e30f});
    const size_t nl = 2 * cands.size();
    std::vector<cudaEvent_t> ev(nl + 1, nullptr);
    Status st;
    for (auto &e : ev) {
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) st = cuda_fail(err, "tuner events");
    }
    if (st.ok()) st = [&]() -> Status {
        TM_CUDA(cudaEventRecord(ev[0], j.st));
        for (size_t i = 0; i < nl; i++) {
            const Cand &c = cands[i % cands.size()];
            j.chunk = c.chunk;
            j.variant = c.variant;
            set_team_shape(j);
            TM_TRY(ensure_order(j));
            TM_TRY(launch_layer_class(j.st, j.L, j.variant, job_layer_params(j), nullptr, nullptr, 0,
                                      j.n_chunks * j.lane_groups));
            TM_CUDA(cudaGetLastError());
            TM_CUDA(cudaEventRecord(ev[i + 1], j.st));
            j.prof->stats.launches++;
        }
        TM_CUDA(cudaEventSynchronize(ev[nl]));
        for (size_t i = 0; i < nl; i++) {
            float ms = 0;
            TM_CUDA(cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
            Cand &c = cands[i % cands.size()];
            c.ms = std::min(c.ms, ms);
        }
        return Status();
    }();
    for (auto e : ev)
        if (e) cudaEventDestroy(e);
    TM_TRY(st);
    const Cand *best = &cands[0];
    for (const Cand &c : cands)
        if (c.ms < best->ms) best = &c;
    {
        std::lock_guard<std::mutex> lock(layer_tune_mutex());
        j.g->layer_tune[j.L] = {best->chunk, best->variant};
    }
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tuned[tune_key(j.L, j.mf)] = {best->chunk, best->variant};
    }
    j.chunk = best->chunk;
    j.variant = best->variant;
    set_team_shape(j);
    std::vector<Job *> one{&j};
    DevBuf unused;
    return launch_layers(j.st, one, unused, nullptr, 0, j.prof);
}

Status job_readout_enqueue(Job &j)
{
    Workspace &w = *j.ws;
    const u64 rows = REDUCE_THREADS / j.L;
    const unsigned blocks = (unsigned)std::max<u64>(1, std::min<u64>((j.n_chunks + rows - 1) / rows,
                                                                     (u64)4 * sm_count()));
    k_reduce_partials<<<blocks, REDUCE_THREADS, 0, j.st>>>(w.partial.as<u64>(), j.n_chunks, j.L, w.out.as<u64>());
    j.prof->stats.launches++;
    TM_CUDA(cudaGetLastError());
    const u64 slot = j.multi_slot ? j.batch_seq : 0;
    TM_CUDA(cudaMemcpyAsync((char *)w.host_pinned + 64 + slot * j.L * 8, w.out.p, (u64)j.L * 8,
                            cudaMemcpyDeviceToHost, j.st));
    return Status();
}

void job_readout_finish(Job &j)
{
    const u64 slot = j.multi_slot ? j.batch_seq : 0;
    const u64 *h_out = (const u64 *)((const char *)j.ws->host_pinned + 64 + slot * j.L * 8);
    const u64 cnt = std::min<u64>(j.L, j.q.p_end - j.p0);
    for (u64 i = 0; i < cnt; i++) {
        j.qsum ^= h_out[i];
        if (j.r == 0) j.vals[j.p0 - j.q.p_begin + i] = h_out[i];
    }
    j.p0 += j.L;
    if (j.p0 < j.q.p_end) return;  // next lane batch of this repeat
    if (j.r == 0) j.sieve_sum = j.qsum;
    if (j.qsum != 0) j.found = 1;
    j.r++;
    j.qsum = 0;
    j.p0 = j.q.p_begin;
    if (j.r >= j.q.repeats) j.done = true;
}

Status job_enqueue_all(Job &j, bool tune)
{
    std::vector<Job *> one{&j};
    DevBuf unused;
    const QuerySpec &q = j.q;
    const u64 nb = (q.p_end - q.p_begin + j.L - 1) / j.L;
    const u64 total = nb * q.repeats;
    TM_TRY(ensure_pinned(*j.ws, 64 + total * j.L * 8));
    j.multi_slot = true;
    // tune only where a layer is long enough for the shape to matter
    // (at least 2^22 arc-lanes, tens of microseconds)
    tune = tune && q.k >= 3 && j.mf * j.L >= (1ull << 22);
    if (tune) {
        std::lock_guard<std::mutex> lock(layer_tune_mutex());
        tune = j.g->layer_tune.find(j.L) == j.g->layer_tune.end();
    }
    for (u64 b = 0; b < total; b++) {
        j.r = (u32)(b / nb);
        j.p0 = q.p_begin + (b % nb) * j.L;
        j.batch_seq = b;
        TM_TRY(job_batch_begin(j));
        for (; j.ell <= q.k; j.ell++) {
            if (tune && b == 0 && j.ell == 3) TM_TRY(tune_layer(j));
            else TM_TRY(launch_layers(j.st, one, unused, nullptr, 0, j.prof));
        }
        TM_TRY(job_readout_enqueue(j));
    }
    return status_take_enqueue(j.st, j.ws->counters.as<u32>() + 12, (u32 *)((char *)j.ws->host_pinned + 48));
}

Status job_finish_all(Job &j)
{
    TM_TRY(status_result(*(const u32 *)((const char *)j.ws->host_pinned + 48)));
    const u64 nb = (j.q.p_end - j.q.p_begin + j.L - 1) / j.L;
    const u64 total = nb * j.q.repeats;
    j.r = 0;
    j.p0 = j.q.p_begin;
    j.qsum = 0;
    for (u64 b = 0; b < total; b++) {
        j.batch_seq = b;
        job_readout_finish(j);
    }
    return Status();
}

Status sieve_decide(Graph &g, const QuerySpec &q, const uint8_t *d_alive, int *found, u64 *sieve_sum,
                    u64 *per_point, double *ms)
{
    Job j;
    j.g = &g;
    j.q = q;
    j.d_alive = d_alive;
    j.ws = &g.ws;
    j.st = g.stream;
    j.prof = &g.prof;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    Status st = [&]() -> Status {
        TM_CUDA(cudaEventCreate(&ev[0]));
        TM_CUDA(cudaEventCreate(&ev[1]));
        TM_CUDA(cudaEventRecord(ev[0], g.stream));
        TM_TRY(job_prep(j));
        if (!j.done) {  // every lane batch of every repeat back to back; one sync at the end
            TM_TRY(job_enqueue_all(j, true));
            TM_CUDA(cudaStreamSynchronize(j.st));
            TM_TRY(job_finish_all(j));
        }
        TM_CUDA(cudaEventRecord(ev[1], g.stream));
        TM_CUDA(cudaEventSynchronize(ev[1]));
        float fms = 0;
        TM_CUDA(cudaEventElapsedTime(&fms, ev[0], ev[1]));
        if (ms) *ms = fms;
        return Status();
    }();
    for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    TM_TRY(st);
    *found = j.found;
    *sieve_sum = j.sieve_sum;
    if (per_point && !j.vals.empty()) std::memcpy(per_point, j.vals.data(), j.vals.size() * sizeof(u64));
    else if (per_point) std::memset(per_point, 0, (q.p_end - q.p_begin) * sizeof(u64));
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

Status gather_arcs(Graph &g, Workspace &w, cudaStream_t st, Profiler &prof, const uint8_t *d_alive, ArcFilter f,
                   std::vector<u32> *src, std::vector<u32> *dst, std::vector<u32> *time)
{
    const u64 m = g.m;
    TM_TRY(w.vflag.reserve(std::max<u64>(g.n, 1)));
    TM_TRY(w.counters.reserve(64));
    k_vflag_mask<<<grid_for(g.n, 256), 256, 0, st>>>(g.n, d_alive, w.vflag.as<uint8_t>());
    prof.stats.launches += 1;
    TM_CUDA(cudaGetLastError());
    u32 *d_cnt = w.counters.as<u32>();
    TM_TRY(filter_arcs_count(st, w, g.d_src, g.d_dst, g.d_time, g.d_in_off, g.n, m, w.vflag.as<uint8_t>(), f, d_cnt,
                             (u64 *)&prof.stats.launches));
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
    TM_TRY(filter_arcs_compact(st, w, g.d_src, g.d_dst, g.d_time, m, w.f_src.as<u32>(), w.f_dst.as<u32>(),
                               w.f_time.as<u32>(), (u64 *)&prof.stats.launches));
    TM_CUDA(cudaMemcpyAsync(src->data(), w.f_src.p, (u64)mf * 4, cudaMemcpyDeviceToHost, st));
    TM_CUDA(cudaMemcpyAsync(dst->data(), w.f_dst.p, (u64)mf * 4, cudaMemcpyDeviceToHost, st));
    TM_CUDA(cudaMemcpyAsync(time->data(), w.f_time.p, (u64)mf * 4, cudaMemcpyDeviceToHost, st));
    TM_CUDA(cudaStreamSynchronize(st));
    return Status();
}

Status make_subgraph(const Graph &g, Workspace &w, cudaStream_t st, const uint8_t *d_alive, Graph *sub)
{
    const u64 m = g.m;
    TM_TRY(w.vflag.reserve(std::max<u64>(g.n, 1)));
    TM_TRY(w.counters.reserve(64));
    k_vflag_mask<<<grid_for(g.n, 256), 256, 0, st>>>(g.n, d_alive, w.vflag.as<uint8_t>());
    TM_CUDA(cudaGetLastError());
    u32 *d_cnt = w.counters.as<u32>();
    TM_TRY(filter_arcs_count(st, w, g.d_src, g.d_dst, g.d_time, g.d_in_off, g.n, m, w.vflag.as<uint8_t>(), ArcFilter(), d_cnt,
                             nullptr));
    u32 mk = 0;
    TM_CUDA(cudaMemcpyAsync(&mk, d_cnt, 4, cudaMemcpyDeviceToHost, st));
    TM_CUDA(cudaStreamSynchronize(st));
    sub->n = g.n;
    sub->m_input = mk;
    sub->m = mk;
    sub->num_colors = g.num_colors;
    sub->max_time = g.max_time;
    sub->stream = st;
    sub->h_color = g.h_color;
    sub->ws.set_stream(st);
    const u64 mb = std::max<u64>(mk, 1) * 4;
    TM_TRY(dev_alloc((void **)&sub->d_src, mb, st));
    TM_TRY(dev_alloc((void **)&sub->d_dst, mb, st));
    TM_TRY(dev_alloc((void **)&sub->d_time, mb, st));
    TM_TRY(dev_alloc((void **)&sub->d_color, std::max<u64>(g.n, 1) * 4, st));
    if (mk) TM_TRY(filter_arcs_compact(st, w, g.d_src, g.d_dst, g.d_time, m, sub->d_src, sub->d_dst, sub->d_time, nullptr));
    TM_CUDA(cudaMemcpyAsync(sub->d_color, g.d_color, (u64)g.n * 4, cudaMemcpyDeviceToDevice, st));
    TM_CUDA(cudaGetLastError());
    sub->resident_bytes = 3 * mb + (u64)g.n * 4;
    return build_in_off(*sub, st, w.block_sums, d_cnt + 15);
}

__global__ void k_first_nonzero(const u64 *sums, u64 mf, u32 *best)
{
    const u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < mf && sums[e]) atomicMin(best, (u32)e);
}

__global__ void k_vertex_sums(const u64 *sums, const u32 *f_dst, u64 mf, u64 *per_vertex)
{
    const u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < mf && sums[e]) atomicXor(&per_vertex[f_dst[e]], sums[e]);
}

// Run one job with arc localisation to the end (all lane batches of its one
// repeat), leaving the arc sums in the graph's workspace.
static Status run_localized(Graph &g, const QuerySpec &q, u32 repeat, const uint8_t *d_alive, Job *jout)
{
    Job &j = *jout;
    j.g = &g;
    j.q = q;
    j.q.repeats = 1;
    j.rep_offset = repeat;
    j.d_alive = d_alive;
    j.ws = &g.ws;
    j.st = g.stream;
    j.prof = &g.prof;
    j.localize = true;
    TM_TRY(job_prep(j));
    if (j.done) return Status();
    std::vector<Job *> one{&j};
    DevBuf unused;
    const u64 nb = (j.q.p_end - j.q.p_begin + j.L - 1) / j.L;
    TM_TRY(ensure_pinned(g.ws, 64 + nb * j.L * 8));
    j.multi_slot = true;
    for (u64 b = 0; b < nb; b++) {
        j.r = 0;
        j.p0 = j.q.p_begin + b * j.L;
        j.batch_seq = b;
        TM_TRY(job_batch_begin(j));
        for (; j.ell <= j.q.k; j.ell++) TM_TRY(launch_layers(j.st, one, unused, nullptr, 0, j.prof));
        TM_TRY(job_readout_enqueue(j));
    }
    return Status();
}

Status job_first_arc(Job &j, u32 *best, u32 *a, u32 *b, u32 *t)
{
    *best = NONE;
    if (j.mf == 0) return Status();
    Workspace &w = *j.ws;
    u32 *d_best = w.counters.as<u32>() + 4;
    TM_CUDA(cudaMemsetAsync(d_best, 0xFF, 4, j.st));
    k_first_nonzero<<<grid_for(j.mf, 256), 256, 0, j.st>>>(w.arc_sum.as<u64>(), j.mf, d_best);
    j.prof->stats.launches++;
    TM_CUDA(cudaGetLastError());
    TM_TRY(ensure_pinned(w));
    u32 *h = (u32 *)((char *)w.host_pinned + 48);
    TM_CUDA(cudaMemcpyAsync(h + 1, d_best, 4, cudaMemcpyDeviceToHost, j.st));
    TM_TRY(status_take_enqueue(j.st, w.counters.as<u32>() + 12, h));
    TM_CUDA(cudaStreamSynchronize(j.st));
    TM_TRY(status_result(h[0]));
    const u32 hb = h[1];
    *best = hb;
    if (hb == NONE) return Status();
    TM_CUDA(cudaMemcpyAsync(a, w.f_src.as<u32>() + hb, 4, cudaMemcpyDeviceToHost, j.st));
    TM_CUDA(cudaMemcpyAsync(b, w.f_dst.as<u32>() + hb, 4, cudaMemcpyDeviceToHost, j.st));
    TM_CUDA(cudaMemcpyAsync(t, w.f_time.as<u32>() + hb, 4, cudaMemcpyDeviceToHost, j.st));
    TM_CUDA(cudaStreamSynchronize(j.st));
    return Status();
}

Status sieve_first_arc(Graph &g, const QuerySpec &q, u32 repeat, const uint8_t *d_alive, u32 *best, u32 *a, u32 *b,
                       u32 *t)
{
    *best = NONE;
    Job j;
    TM_TRY(run_localized(g, q, repeat, d_alive, &j));
    if (j.done) return Status();  // no arc kept
    return job_first_arc(j, best, a, b, t);
}

Status sieve_localize(Graph &g, const QuerySpec &q, u64 *per_vertex, int *found, u64 *sieve_sum, double *ms)
{
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    TM_CUDA(cudaEventCreate(&ev0));
    TM_CUDA(cudaEventCreate(&ev1));
    TM_CUDA(cudaEventRecord(ev0, g.stream));
    Job j;
    TM_TRY(run_localized(g, q, 0, nullptr, &j));
    Workspace &w = g.ws;
    DevBuf pv;
    pv.stream = g.stream;
    TM_TRY(pv.reserve(std::max<u64>(g.n, 1) * 8));
    TM_CUDA(cudaMemsetAsync(pv.p, 0, (u64)g.n * 8, g.stream));
    if (!j.done && j.mf) {
        k_vertex_sums<<<grid_for(j.mf, 256), 256, 0, g.stream>>>(w.arc_sum.as<u64>(), w.f_dst.as<u32>(), j.mf,
                                                                 pv.as<u64>());
        g.prof.stats.launches++;
        TM_CUDA(cudaGetLastError());
    }
    TM_CUDA(cudaMemcpyAsync(per_vertex, pv.p, (u64)g.n * 8, cudaMemcpyDeviceToHost, g.stream));
    TM_CUDA(cudaEventRecord(ev1, g.stream));
    TM_TRY(ensure_pinned(w));
    u32 *h_status = (u32 *)((char *)w.host_pinned + 48);
    TM_TRY(status_take_enqueue(g.stream, w.counters.as<u32>() + 12, h_status));
    TM_CUDA(cudaStreamSynchronize(g.stream));
    TM_TRY(status_result(*h_status));
    pv.release();
    float fms = 0;
    cudaEventElapsedTime(&fms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (ms) *ms = fms;
    u64 s = 0;
    if (!j.done) {
        j.r = 0;
        j.p0 = j.q.p_begin;
        j.qsum = 0;
        const u64 nb = (j.q.p_end - j.q.p_begin + j.L - 1) / j.L;
        for (u64 b = 0; b < nb; b++) {
            j.batch_seq = b;
            job_readout_finish(j);
        }
        s = j.sieve_sum;
    }
    *sieve_sum = s;
    *found = s != 0;
    TM_TRY(g.prof.collect());
    return Status();
}

}  // namespace tmo
