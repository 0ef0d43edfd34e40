// graph.cu -- graph residency built on the device.
//
// E^tau is a set of triples (u, v, j), j >= 1 (Sec. 4).  The build uploads the
// caller's edge arrays and, on the device: validates them, turns each edge
// into one arc (two for undirected input) packed as a 64-bit key
// dst | time | src (bit widths from n and the largest timestamp), marks
// self-loops with a sentinel bit that sorts last, sorts the keys with a
// stable LSD radix sort (8-bit digits, only the bits in use), drops repeated
// keys, and unpacks the arcs into the resident (dst, time, src) order.  When
// dst | time | src needs more than 63 bits, each arc is a pair (time | src,
// dst) instead: a stable sort by time | src and then a stable sort by dst
// give the same order (self-loops get dst = 0xFFFFFFFF, which sorts last).
#include <algorithm>

#include "internal.h"
#include "scan.cuh"

namespace tmo {
namespace {

const int RS_THREADS = 256;
const int RS_PER_THREAD = 16;
const int RS_TILE = RS_THREADS * RS_PER_THREAD;

struct KeySpec {
    int sb, tb, db;  // bits of src, time, dst
    __host__ __device__ int total() const { return sb + tb + db; }
};

__device__ __forceinline__ u64 pack_arc(const KeySpec &ks, u32 dst, u32 t, u32 src)
{
    return ((u64)dst << (ks.tb + ks.sb)) | ((u64)t << ks.sb) | (u64)src;
}

__global__ void k_max_time(u64 m, const u32 *time, u32 *tmax)
{
    u32 best = 0;
    for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (u64)gridDim.x * blockDim.x)
        best = max(best, time[e]);
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) atomicMax(tmax, best);
}

// err bit 1: vertex id >= n; bit 2: timestamp 0; bit 4: colour >= num_colors.
__global__ void k_expand(u64 m, u32 n, const u32 *src, const u32 *dst, const u32 *time, int undirected, KeySpec ks,
                         u64 *keys, u32 *err, unsigned long long *loops)
{
    const u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    const u32 a = src[e], b = dst[e], t = time[e];
    const u64 sentinel = 1ull << ks.total();
    u64 k0 = sentinel, k1 = sentinel;
    if (a >= n || b >= n) atomicOr(err, 1u);
    else if (t == 0) atomicOr(err, 2u);
    else if (a == b) atomicAdd(loops, 1ull);
    else {
        k0 = pack_arc(ks, b, t, a);
        k1 = pack_arc(ks, a, t, b);
    }
    if (undirected) {
        keys[2 * e] = k0;
        keys[2 * e + 1] = k1;
    } else {
        keys[e] = k0;
    }
}

__global__ void k_check_colors(u32 n, const u32 *color, u32 num_colors, u32 *err)
{
    const u64 u = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n && color[u] >= num_colors) atomicOr(err, 4u);
}

// Digit histogram of each tile, stored digit-major: hist[d * ntiles + tile].
template <class K>
__global__ void __launch_bounds__(RS_THREADS) k_radix_hist(const K *keys, u64 N, int shift, u32 ntiles, u32 *hist)
{
    __shared__ u32 h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const u64 base = (u64)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int j = 0; j < RS_PER_THREAD; j++) {
        const u64 i = base + (u64)j * RS_THREADS + threadIdx.x;
        if (i < N) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(u64)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: keys of one tile are ranked in index order (round, warp,
// lane) with warp match groups; offs holds the exclusive digit-major scan.
// With HAS_V each key's value (vin) moves with it.
template <class K, class V, bool HAS_V>
__global__ void __launch_bounds__(RS_THREADS) k_radix_scatter(const K *in, const V *vin, u64 N, int shift,
                                                              u32 ntiles, const u32 *offs, K *out, V *vout)
{
    __shared__ u32 next[256];
    __shared__ u32 wcount[RS_THREADS / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    next[tid] = offs[(u64)tid * ntiles + blockIdx.x];
    for (int i = tid; i < (RS_THREADS / 32) * 256; i += RS_THREADS) (&wcount[0][0])[i] = 0;
    __syncthreads();
    const u64 base = (u64)blockIdx.x * RS_TILE;
    for (int j = 0; j < RS_PER_THREAD; j++) {
        const u64 i = base + (u64)j * RS_THREADS + tid;
        const bool valid = i < N;
        const K key = valid ? in[i] : (K)0;
        const u32 d = valid ? (u32)((key >> shift) & 255u) : 256u;
        const u32 peers = __match_any_sync(0xffffffffu, d);
        const u32 rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wcount[w][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            u32 pre = 0;
            for (int ww = 0; ww < w; ww++) pre += wcount[ww][d];
            out[next[d] + pre + rank] = key;
            if (HAS_V) vout[next[d] + pre + rank] = vin[i];
        }
        __syncthreads();
        u32 tot = 0;
        for (int ww = 0; ww < RS_THREADS / 32; ww++) {
            tot += wcount[ww][tid];
            wcount[ww][tid] = 0;
        }
        next[tid] += tot;
        __syncthreads();
    }
}

// flag[i] = 1 for the first copy of each valid key (keys sorted); flag[N] = 0.
__global__ void k_unique(const u64 *keys, u64 N, u64 sentinel, u32 *flag)
{
    const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > N) return;
    if (i == N) { flag[N] = 0; return; }
    const u64 k = keys[i];
    flag[i] = (k < sentinel && (i == 0 || keys[i - 1] != k)) ? 1u : 0u;
}

// Wide arcs: a = time << sb | src, b = dst (sent, above every vertex id,
// for a self-loop).
__global__ void k_expand_wide(u64 m, u32 n, const u32 *src, const u32 *dst, const u32 *time, int undirected, int sb,
                              u32 sent, u64 *a, u32 *b, u32 *err, unsigned long long *loops)
{
    const u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    const u32 s = src[e], d = dst[e], t = time[e];
    u64 a0 = 0, a1 = 0;
    u32 b0 = sent, b1 = sent;
    if (s >= n || d >= n) atomicOr(err, 1u);
    else if (t == 0) atomicOr(err, 2u);
    else if (s == d) atomicAdd(loops, 1ull);
    else {
        a0 = ((u64)t << sb) | s;
        b0 = d;
        a1 = ((u64)t << sb) | d;
        b1 = s;
    }
    if (undirected) {
        a[2 * e] = a0;
        b[2 * e] = b0;
        a[2 * e + 1] = a1;
        b[2 * e + 1] = b1;
    } else {
        a[e] = a0;
        b[e] = b0;
    }
}

// flag[i] = 1 for the first copy of each arc (sorted pairs); flag[N] = 0.
__global__ void k_unique_wide(const u64 *a, const u32 *b, u64 N, u32 sent, u32 *flag)
{
    const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > N) return;
    if (i == N) { flag[N] = 0; return; }
    flag[i] = (b[i] != sent && (i == 0 || a[i - 1] != a[i] || b[i - 1] != b[i])) ? 1u : 0u;
}

__global__ void k_unpack_wide(const u64 *a, const u32 *b, u64 N, const u32 *off, int sb, u32 *src, u32 *dst,
                              u32 *time)
{
    const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const u32 o = off[i];
    if (off[i + 1] == o) return;
    src[o] = (u32)(a[i] & ((1ull << sb) - 1));
    time[o] = (u32)(a[i] >> sb);
    dst[o] = b[i];
}

__global__ void k_unpack(const u64 *keys, u64 N, const u32 *off, KeySpec ks, u32 *src, u32 *dst, u32 *time)
{
    const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const u32 o = off[i];
    if (off[i + 1] == o) return;
    const u64 k = keys[i];
    src[o] = (u32)(k & ((1ull << ks.sb) - 1));
    time[o] = (u32)((k >> ks.sb) & ((1ull << ks.tb) - 1));
    dst[o] = (u32)(k >> (ks.sb + ks.tb));
}

// Arc counts per (colour of src, colour of dst), for admission estimates.
__global__ void k_color_pairs(u64 m, const u32 *src, const u32 *dst, const u32 *color, u32 nc,
                              unsigned long long *hist)
{
    extern __shared__ unsigned int sh[];
    const u32 bins = nc * nc;
    for (u32 i = threadIdx.x; i < bins; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (u64)gridDim.x * blockDim.x)
        atomicAdd(&sh[color[src[e]] * nc + color[dst[e]]], 1u);
    __syncthreads();
    for (u32 i = threadIdx.x; i < bins; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], (unsigned long long)sh[i]);
}

int bits_for(u64 v)
{
    int b = 1;
    while (b < 64 && (v >> b)) b++;
    return b;
}

unsigned grid(u64 items, int threads) { return (unsigned)std::max<u64>(1, (items + threads - 1) / threads); }

// Scoped device buffer from the library's memory pool.
struct Tmp {
    void *p = nullptr;
    cudaStream_t s;
    explicit Tmp(cudaStream_t st) : s(st) {}
    Status get(size_t bytes) { return dev_alloc(&p, std::max<size_t>(bytes, 16), s); }
    ~Tmp() { if (p) dev_free(p, s); }
    template <class T> T *as() const { return (T *)p; }
};

}  // namespace

// Stable LSD radix sort of N 64-bit keys on their low `bits` bits (8-bit
// digits); a and b are N-key buffers, *sorted points at the one holding the
// result.  d_scratch: one device u32.
Status radix_sort_u64(cudaStream_t st, u64 *a, u64 *b, u64 N, int bits, u32 *d_scratch, u64 **sorted,
                      u64 *launches)
{
    *sorted = a;
    if (N <= 1) return Status();
    const u32 ntiles = (u32)std::max<u64>(1, (N + RS_TILE - 1) / RS_TILE);
    Tmp hist(st);
    DevBuf tiles;
    tiles.stream = st;
    TM_TRY(hist.get((u64)256 * ntiles * 4));
    for (int shift = 0; shift < bits; shift += 8) {
        k_radix_hist<u64><<<ntiles, RS_THREADS, 0, st>>>(a, N, shift, ntiles, hist.as<u32>());
        TM_TRY(exclusive_scan_on(st, tiles, hist.as<u32>(), (u64)256 * ntiles, d_scratch, launches));
        k_radix_scatter<u64, u64, false>
            <<<ntiles, RS_THREADS, 0, st>>>(a, nullptr, N, shift, ntiles, hist.as<u32>(), b, nullptr);
        TM_CUDA(cudaGetLastError());
        if (launches) *launches += 2;
        std::swap(a, b);
    }
    tiles.release();
    *sorted = a;
    return Status();
}

namespace {

// Stable LSD radix sort of N keys (K) with values (V) on the keys' low
// `bits` bits; (*k, *v) point at the buffers holding the result.
template <class K, class V>
Status radix_sort_pairs(cudaStream_t st, K *ka, K *kb, V *va, V *vb, u64 N, int bits, u32 *d_scratch, K **k,
                        V **v, u64 *launches)
{
    *k = ka;
    *v = va;
    if (N <= 1) return Status();
    const u32 ntiles = (u32)std::max<u64>(1, (N + RS_TILE - 1) / RS_TILE);
    Tmp hist(st);
    DevBuf tiles;
    tiles.stream = st;
    TM_TRY(hist.get((u64)256 * ntiles * 4));
    for (int shift = 0; shift < bits; shift += 8) {
        k_radix_hist<K><<<ntiles, RS_THREADS, 0, st>>>(ka, N, shift, ntiles, hist.as<u32>());
        TM_TRY(exclusive_scan_on(st, tiles, hist.as<u32>(), (u64)256 * ntiles, d_scratch, launches));
        k_radix_scatter<K, V, true><<<ntiles, RS_THREADS, 0, st>>>(ka, va, N, shift, ntiles, hist.as<u32>(), kb, vb);
        TM_CUDA(cudaGetLastError());
        if (launches) *launches += 2;
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    tiles.release();
    *k = ka;
    *v = va;
    return Status();
}

}  // namespace

Status build_graph_device(const tmotif_graph_desc *d, Graph *g)
{
    cudaStream_t st = (cudaStream_t)d->cuda_stream;
    const u64 m = d->m;
    const int und = d->undirected ? 1 : 0;
    const u64 N = und ? 2 * m : m;
    const u32 n = d->n;

    Tmp raw(st), small(st), keys(st), keys2(st), flag(st), hist(st);
    DevBuf tiles;
    tiles.stream = st;
    TM_TRY(small.get(256));
    u32 *d_small = small.as<u32>();  // [0] max time, [1] err, [2] arc count, [4..5] loops (u64)
    TM_CUDA(cudaMemsetAsync(d_small, 0, 256, st));
    TM_TRY(raw.get(std::max<u64>(3 * m, 1) * 4 + (u64)std::max<u32>(n, 1) * 4));
    u32 *r_src = raw.as<u32>(), *r_dst = r_src + m, *r_time = r_dst + m, *r_color = r_time + m;
    if (m) {
        TM_CUDA(cudaMemcpyAsync(r_src, d->src, m * 4, cudaMemcpyHostToDevice, st));
        TM_CUDA(cudaMemcpyAsync(r_dst, d->dst, m * 4, cudaMemcpyHostToDevice, st));
        TM_CUDA(cudaMemcpyAsync(r_time, d->time, m * 4, cudaMemcpyHostToDevice, st));
        k_max_time<<<std::min<unsigned>(grid(m, 256), 1024), 256, 0, st>>>(m, r_time, d_small + 0);
    }
    TM_CUDA(cudaMemcpyAsync(r_color, d->color, (u64)n * 4, cudaMemcpyHostToDevice, st));
    k_check_colors<<<grid(n, 256), 256, 0, st>>>(n, r_color, d->num_colors, d_small + 1);
    TM_CUDA(cudaGetLastError());
    u32 h[2] = {0, 0};
    TM_CUDA(cudaMemcpyAsync(h, d_small, 8, cudaMemcpyDeviceToHost, st));
    TM_CUDA(cudaStreamSynchronize(st));
    if (h[1] & 4u) return fail(TMOTIF_ERR_INVALID, "color out of range");
    const u32 tmax = h[0];
    KeySpec ks;
    ks.sb = ks.db = bits_for(n > 0 ? n - 1 : 0);
    ks.tb = bits_for(tmax);
    // dst | time | src plus the sentinel bit in one 64-bit key, else pairs
    const bool wide = ks.total() + 1 > 64;
    const u32 sent = ks.db < 32 ? (1u << ks.db) : NONE;  // wide sentinel dst
    const int bits_b = ks.db < 32 ? ks.db + 1 : 32;
    Tmp vals(st), vals2(st);

    TM_TRY(keys.get(N * 8));
    TM_TRY(keys2.get(N * 8));
    if (wide) {
        TM_TRY(vals.get(N * 4));
        TM_TRY(vals2.get(N * 4));
    }
    if (m) {
        if (wide)
            k_expand_wide<<<grid(m, 256), 256, 0, st>>>(m, n, r_src, r_dst, r_time, und, ks.sb, sent, keys.as<u64>(),
                                                        vals.as<u32>(), d_small + 1,
                                                        (unsigned long long *)(d_small + 4));
        else
            k_expand<<<grid(m, 256), 256, 0, st>>>(m, n, r_src, r_dst, r_time, und, ks, keys.as<u64>(), d_small + 1,
                                                   (unsigned long long *)(d_small + 4));
        TM_CUDA(cudaGetLastError());
    }
    u64 hl[3] = {0, 0, 0};
    TM_CUDA(cudaMemcpyAsync(hl, d_small, 24, cudaMemcpyDeviceToHost, st));
    TM_CUDA(cudaStreamSynchronize(st));
    const u32 err = ((u32 *)hl)[1];
    if (err & 1u) return fail(TMOTIF_ERR_INVALID, "vertex id out of range");
    if (err & 2u) return fail(TMOTIF_ERR_INVALID, "timestamp 0 (timestamps are >= 1)");
    const u64 loops = hl[2];

    // LSD radix sort over the bits in use plus the sentinel bit (wide: by
    // time | src, then stably by dst).
    u64 *a = nullptr;
    u32 *b = nullptr;
    u64 launches = 0;
    if (wide) {
        u64 *a1 = nullptr;
        u32 *b1 = nullptr;
        TM_TRY(radix_sort_pairs(st, keys.as<u64>(), keys2.as<u64>(), vals.as<u32>(), vals2.as<u32>(), N,
                                          ks.tb + ks.sb, d_small + 2, &a1, &b1, &launches));
        u64 *a2 = a1 == keys.as<u64>() ? keys2.as<u64>() : keys.as<u64>();
        u32 *b2 = b1 == vals.as<u32>() ? vals2.as<u32>() : vals.as<u32>();
        TM_TRY(radix_sort_pairs(st, b1, b2, a1, a2, N, bits_b, d_small + 2, &b, &a, &launches));
    } else {
        TM_TRY(radix_sort_u64(st, keys.as<u64>(), keys2.as<u64>(), N, ks.total() + 1, d_small + 2, &a, &launches));
    }
    // dedupe (E^tau is a set), drop sentinels, unpack
    TM_TRY(flag.get((N + 1) * 4));
    if (wide)
        k_unique_wide<<<grid(N + 1, 256), 256, 0, st>>>(a, b, N, sent, flag.as<u32>());
    else
        k_unique<<<grid(N + 1, 256), 256, 0, st>>>(a, N, 1ull << ks.total(), flag.as<u32>());
    TM_TRY(exclusive_scan_on(st, tiles, flag.as<u32>(), N + 1, d_small + 2, &launches));
    u32 mk = 0;
    TM_CUDA(cudaMemcpyAsync(&mk, d_small + 2, 4, cudaMemcpyDeviceToHost, st));
    TM_CUDA(cudaStreamSynchronize(st));
    const u64 mb = std::max<u64>(mk, 1) * 4;
    TM_TRY(dev_alloc((void **)&g->d_src, mb, st));
    TM_TRY(dev_alloc((void **)&g->d_dst, mb, st));
    TM_TRY(dev_alloc((void **)&g->d_time, mb, st));
    TM_TRY(dev_alloc((void **)&g->d_color, (u64)std::max<u32>(n, 1) * 4, st));
    if (N && wide)
        k_unpack_wide<<<grid(N, 256), 256, 0, st>>>(a, b, N, flag.as<u32>(), ks.sb, g->d_src, g->d_dst, g->d_time);
    else if (N)
        k_unpack<<<grid(N, 256), 256, 0, st>>>(a, N, flag.as<u32>(), ks, g->d_src, g->d_dst, g->d_time);
    TM_CUDA(cudaMemcpyAsync(g->d_color, r_color, (u64)n * 4, cudaMemcpyDeviceToDevice, st));
    TM_CUDA(cudaGetLastError());
    g->pair_hist.clear();
    const u32 nc = d->num_colors;
    if (nc <= PAIR_HIST_COLORS && mk > 0) {
        TM_TRY(hist.get((u64)nc * nc * 8));
        TM_CUDA(cudaMemsetAsync(hist.p, 0, (u64)nc * nc * 8, st));
        k_color_pairs<<<std::min<unsigned>(grid(mk, 256), 1024), 256, (size_t)nc * nc * 4, st>>>(
            mk, g->d_src, g->d_dst, g->d_color, nc, (unsigned long long *)hist.p);
        TM_CUDA(cudaGetLastError());
        g->pair_hist.assign((size_t)nc * nc, 0);
        TM_CUDA(cudaMemcpyAsync(g->pair_hist.data(), hist.p, (u64)nc * nc * 8, cudaMemcpyDeviceToHost, st));
    }
    g->n = n;
    g->m = mk;
    TM_TRY(build_in_off(*g, st, tiles, d_small + 8));
    TM_CUDA(cudaStreamSynchronize(st));
    tiles.release();

    g->m_input = m;
    g->self_loops = loops;
    g->duplicates = (m - loops) * (und ? 2 : 1) - mk;
    g->num_colors = d->num_colors;
    g->max_time = tmax;
    g->stream = st;
    g->resident_bytes += 3 * mb + (u64)std::max<u32>(n, 1) * 4;
    return Status();
}

}  // namespace tmo
