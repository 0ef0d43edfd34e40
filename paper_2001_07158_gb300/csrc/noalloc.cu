// noalloc.cu -- a decision that allocates no memory: tmotif_decide_noalloc.
//
// Some callers cannot allocate device memory at the moment they need an
// answer: a host program whose own allocator already owns the whole device,
// a latency-critical loop where cudaMalloc/cudaFree would synchronise the
// device, or code running under a fixed memory budget set elsewhere.  This
// entry point serves them: the caller passes the graph and the output buffer
// (device memory it owns) and all intermediate data lives in one file-scope
// device array of fixed size, TMOTIF_NOALLOC_SCRATCH_BYTES, which every GPU
// that loads the library keeps until the process exits.
//
// The array is shared by every call and keeps the previous call's contents;
// each call clears what must start at zero.  Two calls whose work overlaps on
// the GPU (different streams, or different host threads on one device) race
// on the array and give wrong answers: serialise them.
//
// In host code the array's name is only a host-side stand-in; its device
// address comes from cudaGetSymbolAddress, looked up once per device by the
// first call made on that device (with that device current).  Make that first
// call before any stream capture.  The looked-up address is kept for the life
// of the process: after a cudaDeviceReset of a device, this entry point must
// not be called on that device again.  Every call synchronises its stream
// before it returns (it reads a validation flag and waits for the result).
#include <mutex>

#include "gf64.cuh"
#include "internal.h"

namespace tmo {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[TMOTIF_NOALLOC_SCRATCH_BYTES];

const u32 NA_LANES = 64;     // lane width of every batch (one warp per arc team)
const u32 NA_CHUNK = 128;    // arcs per team chunk (whole in-segments)
const u32 NA_COLORS_MAX = 4096;

// Byte offsets of the pieces of the scratch array for one call.
struct Layout {
    size_t err, cnt, slot_count, slot_begin, keep, f_src, f_dst, f_time, pos, mark, cp_in, cp_out, seg_lo, seg_hi,
        wtab, out, x, c0, c1, total;
};

size_t up(size_t v) { return (v + 255) & ~(size_t)255; }

Layout layout_for(u32 n, u64 m, u32 num_colors, u32 k)
{
    Layout l;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o += up(bytes); return at; };
    l.err = take(4);
    l.cnt = take(16);
    l.slot_count = take((size_t)num_colors * 4);
    l.slot_begin = take((size_t)num_colors * 4);
    l.keep = take((m + 1) * 4);
    l.f_src = take(m * 4);
    l.f_dst = take(m * 4);
    l.f_time = take(m * 4);
    l.pos = take(m * 4);
    l.mark = take((m + 1) * 4);
    l.cp_in = take(m * 4);
    l.cp_out = take(m * 4);
    l.seg_lo = take((size_t)n * 4);
    l.seg_hi = take((size_t)n * 4);
    l.wtab = take((size_t)k * NA_LANES * 8);
    l.out = take(NA_LANES * 8);
    l.x = take((size_t)n * NA_LANES * 8);
    l.c0 = take(m * NA_LANES * 8);  // checkpoints are at most the kept arcs
    l.c1 = take(m * NA_LANES * 8);
    l.total = o;
    return l;
}

// Every vertex colour must be < num_colors (the coefficient kernel indexes
// the slot tables by the colour of every vertex, with or without arcs).
__global__ void k_na_check_colors(u32 n, const u32 *color, u32 num_colors, u32 *err)
{
    const u64 u = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n && color[u] >= num_colors) atomicOr(err, 2u);
}

// Arcs must be canonical: ids < n, time >= 1, no self-loop, strictly
// increasing in (dst, time, src) order.  Also marks the arcs to keep.
__global__ void k_na_check_keep(u64 m, u32 n, const u32 *src, const u32 *dst, const u32 *time, const u32 *color,
                                u32 num_colors, const u32 *slot_count, u32 t_min, u32 t_max, u32 *keep, u32 *err)
{
    u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (e > m) return;
    if (e == m) { keep[m] = 0; return; }
    const u32 a = src[e], b = dst[e], t = time[e];
    bool bad = a >= n || b >= n || t == 0 || a == b;
    if (!bad && e > 0) {
        const u32 pb = dst[e - 1], pt = time[e - 1], pa = src[e - 1];
        const bool inc = pb < b || (pb == b && (pt < t || (pt == t && pa < a)));
        bad = !inc;
    }
    if (bad) {
        atomicOr(err, 1u);
        keep[e] = 0;
        return;
    }
    const u32 ca = color[a], cb = color[b];
    bad = ca >= num_colors || cb >= num_colors;
    if (bad) {
        atomicOr(err, 1u);
        keep[e] = 0;
        return;
    }
    keep[e] = (slot_count[ca] && slot_count[cb] && t >= t_min && (t_max == 0 || t <= t_max)) ? 1u : 0u;
}

// Exclusive scan of a[0..N) in place by one block; total to *total.
__global__ void __launch_bounds__(1024) k_na_scan(u32 *a, const u32 *N_ptr, u64 N_fixed, u32 *total)
{
    __shared__ u32 part[1024];
    const u64 N = N_ptr ? (u64)(*N_ptr) + 1 : N_fixed;
    const u64 per = (N + blockDim.x - 1) / blockDim.x;
    const u64 b = threadIdx.x * per, e = min(N, b + per);
    u32 s = 0;
    for (u64 i = b; i < e; i++) s += a[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (u32 o = 1; o < blockDim.x; o <<= 1) {
        u32 v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    u32 run = part[threadIdx.x] - s;
    for (u64 i = b; i < e; i++) {
        u32 v = a[i];
        a[i] = run;
        run += v;
    }
    if (threadIdx.x == blockDim.x - 1) *total = part[threadIdx.x];
}

__global__ void k_na_compact(u64 m, const u32 *src, const u32 *dst, const u32 *time, const u32 *off, u32 *f_src,
                             u32 *f_dst, u32 *f_time)
{
    u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    const u32 o = off[e];
    if (off[e + 1] != o) {
        f_src[o] = src[e];
        f_dst[o] = dst[e];
        f_time[o] = time[e];
    }
}

__global__ void k_na_segments(const u32 *mf_ptr, const u32 *f_dst, u32 *seg_lo, u32 *seg_hi)
{
    const u64 mf = *mf_ptr;
    u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= mf) return;
    const u32 d = f_dst[e];
    if (e == 0 || f_dst[e - 1] != d) seg_lo[d] = (u32)e;
    if (e + 1 == mf || f_dst[e + 1] != d) seg_hi[d] = (u32)(e + 1);
}

// Last in-arc of src(e) with an earlier time (strictly increasing times).
__global__ void k_na_pos(const u32 *mf_ptr, const u32 *f_src, const u32 *f_time, const u32 *seg_lo,
                         const u32 *seg_hi, u32 *pos, u32 *mark)
{
    const u64 mf = *mf_ptr;
    u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= mf) return;
    const u32 a = f_src[e], t = f_time[e];
    u32 lo = seg_lo[a], hi = seg_hi[a];
    const u32 first = lo;
    while (lo < hi) {
        const u32 mid = lo + ((hi - lo) >> 1);
        if (f_time[mid] < t) lo = mid + 1;
        else hi = mid;
    }
    u32 p = NONE;
    if (lo > first) {
        p = lo - 1;
        mark[p] = 1;
    }
    pos[e] = p;
}

__global__ void k_na_checkpoints(const u32 *mf_ptr, const u32 *pos, const u32 *ck, u32 *cp_in, u32 *cp_out)
{
    const u64 mf = *mf_ptr;
    u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= mf) return;
    const u32 p = pos[e];
    cp_in[e] = (p == NONE) ? NONE : ck[p];
    cp_out[e] = (ck[e + 1] != ck[e]) ? ck[e] : NONE;
}

__global__ void k_na_wtab(u32 k, u64 p0, QueryKeys keys, u64 *wtab)
{
    const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k * NA_LANES) return;
    const u32 d = i / NA_LANES;
    const u64 point = p0 + i % NA_LANES;
    u64 s = 0;
    for (u32 j = 0; j < k; j++)
        if ((point >> j) & 1u) s ^= coef_w(keys, d, j);
    wtab[i] = s;
}

__global__ void k_na_coef(u32 n, const u32 *color, const u32 *slot_begin, const u32 *slot_count, QueryKeys keys,
                          const u64 *wtab, u64 *x)
{
    const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (u64)n * NA_LANES) return;
    const u32 u = (u32)(i / NA_LANES), lane = (u32)(i % NA_LANES);
    const u32 c = color[u];
    const u32 d0 = slot_begin[c], d1 = d0 + slot_count[c];
    u64 s = 0;
    for (u32 d = d0; d < d1; d++) s ^= gf_mul(coef_v(keys, u, d), wtab[(u64)d * NA_LANES + lane]);
    x[i] = s;
}

// One layer of eq. (gen-polynomial:3): a warp owns the 64 lanes of a chunk of
// whole in-segments (2 lanes per thread), as in the main layer kernel.
__global__ void __launch_bounds__(256) k_na_layer(const u32 *mf_ptr, const u32 *src, const u32 *dst, const u32 *time,
                                                  const u32 *cp_in, const u32 *cp_out, const u32 *seg_hi,
                                                  const u64 *x, const u64 *Cin, u64 *Cout, u64 *out, u64 ky, u32 ell,
                                                  u32 k, u32 start, u32 end)
{
    const u64 mf = *mf_ptr;
    const int tt = threadIdx.x & 31;
    const u64 chunk = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const u32 lane0 = 2 * tt;
    u64 q0 = 0, q1 = 0;
    const u64 b0 = chunk * NA_CHUNK;
    if (b0 < mf) {
        const u64 b1 = min(b0 + NA_CHUNK, mf);
        u64 begin = b0, stop = b1;
        if (b0 > 0 && dst[b0] == dst[b0 - 1]) begin = seg_hi[dst[b0]];
        if (b1 < mf && dst[b1] == dst[b1 - 1]) stop = seg_hi[dst[b1]];
        const bool last = (ell == k);
        u32 cur = NONE;
        u64 xc0 = 0, xc1 = 0, acc0 = 0, acc1 = 0;
        for (u64 e = begin; e < stop; e++) {
            const u32 s = src[e], d = dst[e];
            if (d != cur) {
                if (last && cur != NONE && (end == NONE || cur == end)) {
                    q0 ^= gf_mul(xc0, acc0);
                    q1 ^= gf_mul(xc1, acc1);
                }
                cur = d;
                acc0 = acc1 = 0;
                xc0 = x[(u64)d * NA_LANES + lane0];
                xc1 = x[(u64)d * NA_LANES + lane0 + 1];
            }
            const u64 y = coef_y(mix64(ky ^ (((u64)s << 32) | d)), time[e], ell - 1);
            const u64 *in = nullptr;
            if (ell == 2) {
                if (start == NONE || s == start) in = x + (u64)s * NA_LANES;
            } else {
                const u32 ci = cp_in[e];
                if (ci != NONE) in = Cin + (u64)ci * NA_LANES;
            }
            if (in) {
                acc0 ^= gf_mul(y, in[lane0]);
                acc1 ^= gf_mul(y, in[lane0 + 1]);
            }
            if (!last) {
                const u32 co = cp_out[e];
                if (co != NONE) {
                    Cout[(u64)co * NA_LANES + lane0] = gf_mul(xc0, acc0);
                    Cout[(u64)co * NA_LANES + lane0 + 1] = gf_mul(xc1, acc1);
                }
            }
        }
        if (last && cur != NONE && (end == NONE || cur == end)) {
            q0 ^= gf_mul(xc0, acc0);
            q1 ^= gf_mul(xc1, acc1);
        }
    }
    if (ell == k) {
        if (q0) atomicXor(&out[lane0], q0);
        if (q1) atomicXor(&out[lane0 + 1], q1);
    }
}

std::mutex g_na_mutex;
void *g_na_ptr[256];  // device address of the scratch array, per device

Status scratch_address(void **ptr)
{
    int dev = 0;
    TM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return fail(TMOTIF_ERR_UNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        TM_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_na_ptr[dev] = p;
    }
    *ptr = g_na_ptr[dev];
    return Status();
}

unsigned blocks_for(u64 items, int threads) { return (unsigned)((items + threads - 1) / threads); }

Status decide_noalloc(const u32 *src, const u32 *dst, const u32 *time, u64 m, const u32 *color, u32 n,
                      u32 num_colors, const tmotif_query *q, u64 *d_out, cudaStream_t st)
{
    if (!q || !q->multiset) return fail(TMOTIF_ERR_INVALID, "null query");
    if (q->k < 2 || q->k > TMOTIF_KMAX) return fail(TMOTIF_ERR_UNSUPPORTED, "k must be in [2, 20]");
    if (q->repeats != 1) return fail(TMOTIF_ERR_INVALID, "the allocation-free decision evaluates one repeat");
    if (q->timestamps) return fail(TMOTIF_ERR_UNSUPPORTED, "the allocation-free decision takes no EC timestamps");
    if (num_colors == 0 || num_colors > NA_COLORS_MAX) return fail(TMOTIF_ERR_INVALID, "num_colors must be in [1, 4096]");
    if (n == 0 || (m > 0 && (!src || !dst || !time)) || !color || !d_out)
        return fail(TMOTIF_ERR_INVALID, "null graph or output pointer");
    // arc offsets, counts and checkpoint numbers are 32-bit (and the scratch
    // layout below is computed in size_t, which this bound keeps exact)
    if (m > (u64)0xFFFFFFFEu) return fail(TMOTIF_ERR_INVALID, "m must be below 2^32 - 1");
    if (q->start != TMOTIF_ANY && q->start >= n) return fail(TMOTIF_ERR_INVALID, "start vertex out of range");
    if (q->end != TMOTIF_ANY && q->end >= n) return fail(TMOTIF_ERR_INVALID, "end vertex out of range");
    const u32 k = q->k;
    const u64 full = 1ull << k;
    u64 p_begin = 0, p_end = full;
    if (q->point_begin != 0 || q->point_end != 0) {
        if (q->point_begin >= q->point_end || q->point_end > full) return fail(TMOTIF_ERR_INVALID, "bad point range");
        p_begin = q->point_begin;
        p_end = q->point_end;
    }
    u32 slot_count[NA_COLORS_MAX] = {0}, slot_begin[NA_COLORS_MAX] = {0};
    for (u32 r = 0; r < k; r++) {
        if (q->multiset[r] >= num_colors) return fail(TMOTIF_ERR_INVALID, "multiset colour out of range");
        slot_count[q->multiset[r]]++;
    }
    for (u32 c = 0, off = 0; c < num_colors; c++) { slot_begin[c] = off; off += slot_count[c]; }

    const Layout L = layout_for(n, m, num_colors, k);
    if (L.total > TMOTIF_NOALLOC_SCRATCH_BYTES)
        return fail(TMOTIF_ERR_UNSUPPORTED, "graph too large for the allocation-free decision: needs " +
                                                std::to_string(L.total) + " bytes of scratch, the fixed array has " +
                                                std::to_string((u64)TMOTIF_NOALLOC_SCRATCH_BYTES));
    void *base = nullptr;
    TM_TRY(scratch_address(&base));
    unsigned char *S = (unsigned char *)base;
    u32 *err = (u32 *)(S + L.err), *cnt = (u32 *)(S + L.cnt);
    u32 *d_slot_count = (u32 *)(S + L.slot_count), *d_slot_begin = (u32 *)(S + L.slot_begin);
    u32 *keep = (u32 *)(S + L.keep), *f_src = (u32 *)(S + L.f_src), *f_dst = (u32 *)(S + L.f_dst);
    u32 *f_time = (u32 *)(S + L.f_time), *pos = (u32 *)(S + L.pos), *mark = (u32 *)(S + L.mark);
    u32 *cp_in = (u32 *)(S + L.cp_in), *cp_out = (u32 *)(S + L.cp_out);
    u32 *seg_lo = (u32 *)(S + L.seg_lo), *seg_hi = (u32 *)(S + L.seg_hi);
    u64 *wtab = (u64 *)(S + L.wtab), *out = (u64 *)(S + L.out), *x = (u64 *)(S + L.x);
    u64 *C[2] = {(u64 *)(S + L.c0), (u64 *)(S + L.c1)};

    // Validate the colours and the arcs and pick the arcs whose colours are in
    // the multiset.
    TM_CUDA(cudaMemsetAsync(err, 0, 4, st));
    TM_CUDA(cudaMemsetAsync(cnt, 0, 16, st));
    TM_CUDA(cudaMemcpyAsync(d_slot_count, slot_count, num_colors * 4, cudaMemcpyHostToDevice, st));
    TM_CUDA(cudaMemcpyAsync(d_slot_begin, slot_begin, num_colors * 4, cudaMemcpyHostToDevice, st));
    k_na_check_colors<<<blocks_for(n, 256), 256, 0, st>>>(n, color, num_colors, err);
    k_na_check_keep<<<blocks_for(m + 1, 256), 256, 0, st>>>(m, n, src, dst, time, color, num_colors, d_slot_count,
                                                            q->t_min, q->t_max, keep, err);
    TM_CUDA(cudaGetLastError());
    u32 h_err = 0;
    TM_CUDA(cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, st));
    TM_CUDA(cudaStreamSynchronize(st));
    if (h_err & 2u) return fail(TMOTIF_ERR_INVALID, "every vertex colour must be < num_colors");
    if (h_err)
        return fail(TMOTIF_ERR_INVALID, "arcs must have ids < n, time >= 1, no self-loops, colours < num_colors, "
                                        "and be strictly increasing in (dst, time, src)");
    if (m == 0) {  // no arcs, no walks: every per-point sum is zero
        TM_CUDA(cudaMemsetAsync(d_out, 0, (p_end - p_begin) * 8, st));
        TM_CUDA(cudaStreamSynchronize(st));
        return Status();
    }

    // Compact, segments, last earlier in-arc, checkpoints (counts stay on the device).
    k_na_scan<<<1, 1024, 0, st>>>(keep, nullptr, m + 1, cnt + 0);
    k_na_compact<<<blocks_for(m, 256), 256, 0, st>>>(m, src, dst, time, keep, f_src, f_dst, f_time);
    TM_CUDA(cudaMemsetAsync(seg_lo, 0, (size_t)n * 4, st));
    TM_CUDA(cudaMemsetAsync(seg_hi, 0, (size_t)n * 4, st));
    TM_CUDA(cudaMemsetAsync(mark, 0, (m + 1) * 4, st));
    k_na_segments<<<blocks_for(m, 256), 256, 0, st>>>(cnt + 0, f_dst, seg_lo, seg_hi);
    k_na_pos<<<blocks_for(m, 256), 256, 0, st>>>(cnt + 0, f_src, f_time, seg_lo, seg_hi, pos, mark);
    k_na_scan<<<1, 1024, 0, st>>>(mark, cnt + 0, 0, cnt + 1);
    k_na_checkpoints<<<blocks_for(m, 256), 256, 0, st>>>(cnt + 0, pos, mark, cp_in, cp_out);
    TM_CUDA(cudaGetLastError());

    // Lane batches of 64 points: coefficients, layers 2..k, per-point sums.
    const QueryKeys keys = make_keys(mix64(q->seed + TM_GOLDEN));
    const u64 teams = (m + NA_CHUNK - 1) / NA_CHUNK;
    for (u64 p0 = p_begin; p0 < p_end; p0 += NA_LANES) {
        const u64 count = (p_end - p0 < NA_LANES) ? p_end - p0 : NA_LANES;
        k_na_wtab<<<blocks_for((u64)k * NA_LANES, 128), 128, 0, st>>>(k, p0, keys, wtab);
        k_na_coef<<<blocks_for((u64)n * NA_LANES, 256), 256, 0, st>>>(n, color, d_slot_begin, d_slot_count, keys,
                                                                     wtab, x);
        TM_CUDA(cudaMemsetAsync(out, 0, NA_LANES * 8, st));
        for (u32 ell = 2; ell <= k; ell++)
            k_na_layer<<<blocks_for(teams * 32, 256), 256, 0, st>>>(cnt + 0, f_src, f_dst, f_time, cp_in, cp_out,
                                                                    seg_hi, x, C[ell & 1], C[(ell + 1) & 1], out,
                                                                    keys.ky, ell, k, q->start, q->end);
        TM_CUDA(cudaGetLastError());
        TM_CUDA(cudaMemcpyAsync(d_out + (p0 - p_begin), out, count * 8, cudaMemcpyDeviceToDevice, st));
    }
    TM_CUDA(cudaStreamSynchronize(st));
    return Status();
}

}  // namespace
}  // namespace tmo

extern "C" int tmotif_decide_noalloc(const uint32_t *d_src, const uint32_t *d_dst, const uint32_t *d_time,
                                     uint64_t m, const uint32_t *d_color, uint32_t n, uint32_t num_colors,
                                     const tmotif_query *q, uint64_t *d_per_point, void *cuda_stream)
{
    return tmo::decide_noalloc(d_src, d_dst, d_time, m, d_color, n, num_colors, q, (tmo::u64 *)d_per_point,
                               (cudaStream_t)cuda_stream)
        .code;
}
