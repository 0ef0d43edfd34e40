// scan.cuh -- exclusive prefix sums of u32 arrays on the device (three
// phases: tile sums, one-block scan of the tile sums, tile scan).  Totals fit
// in u32 because arc counts are below 2^32.  Included by the translation units
// that need it; the kernels are file-local.
#pragma once
#include "internal.h"

namespace tmo {
namespace {

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


// In-place exclusive scan of a[0..N) on `stream`; the total goes to d_total
// (device u32).  `tiles` is a device buffer grown as needed.
inline Status exclusive_scan_on(cudaStream_t stream, DevBuf &tiles, u32 *a, u64 N, u32 *d_total, u64 *launches)
{
    u64 ntiles = (N + SCAN_TILE - 1) / SCAN_TILE;
    if (ntiles == 0) ntiles = 1;
    TM_TRY(tiles.reserve(ntiles * sizeof(u32)));
    u32 *sums = tiles.as<u32>();
    k_tile_sum<<<(unsigned)ntiles, SCAN_THREADS, 0, stream>>>(a, N, sums);
    k_scan_tiles<<<1, 1024, 0, stream>>>(sums, (u32)ntiles, d_total);
    k_tile_scan<<<(unsigned)ntiles, SCAN_THREADS, 0, stream>>>(a, N, sums, a);
    if (launches) *launches += 3;
    TM_CUDA(cudaGetLastError());
    return Status();
}

}  // namespace
}  // namespace tmo
