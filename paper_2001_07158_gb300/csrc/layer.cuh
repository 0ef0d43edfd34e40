// layer.cuh -- the team body of the generating-function layer kernel
// (eq. gen-polynomial:3), shared by the per-query kernels (sieve.cu) and the
// packed many-graph batch (pack.cu).
#pragma once
#include "gf64.cuh"
#include "internal.h"

namespace tmo {

// ---------------------------------------------------------------------------
// A team of T threads owns T * LPT consecutive lanes (LPT = 1, 2 or 4 lanes,
// 8, 16 or 32 bytes, per thread) of one job and walks one chunk of whole
// in-segments in arc order: team index = chunk * lane_groups + lane group.
// A resident team calls this once for every team index it takes from its
// launch's counter.  Segments are never split, so a running XOR is
// the prefix of eq. (3)'s stay term.  With TAB the team builds, per arc, the
// nibble table of y_{e,l-1} in shared memory and every lane's y-product is 16
// table loads; x-products (one per checkpoint and per segment at the last
// layer) use the register multiply.  At the last layer every team writes its
// lanes' sums to the job's partial array.
//
// PACKED: the arcs of many small graphs with their own queries, packed with
// vertex ids offset per graph (pack.cu).  A segment's job is its destination's
// (p.jv); y uses the job's key and the graph's own vertex ids; the job's own
// k decides whether this layer is past its end (segment skipped), its last
// (segment sums XORed into the job's lane sums p.pout) or an inner layer.
//
// INNER: the caller guarantees 2 < l < k (single job), so the form for the
// first and the last layer (source rows from x, segment sums) compiles out.
// ---------------------------------------------------------------------------
template <int T, bool TAB, int LPT, bool PACKED, bool INNER = false>
__device__ __forceinline__ void layer_team(const LayerParams &p, u64 team, u64 *tab)
{
    const int tt = threadIdx.x % T;
    const u32 team_mask = (T == 32) ? 0xffffffffu : (((1u << T) - 1u) << (((threadIdx.x & 31) / T) * T));
    const u64 chunk = team / p.lane_groups;
    if (chunk >= p.n_chunks) return;
    const u32 lane0 = (u32)(team % p.lane_groups) * (LPT * T) + LPT * tt;
    const u64 Lw = p.L;
    const bool last = !PACKED && !INNER && (p.ell == p.k);
    u64 q[LPT], xc[LPT], acc[LPT];
#pragma unroll
    for (int i = 0; i < LPT; i++) q[i] = xc[i] = acc[i] = 0;

    const u64 b0 = chunk * p.chunk;
    const u64 b1 = min(b0 + p.chunk, p.m_f);
    u64 begin = b0, stop = b1;
    if (b0 > 0 && p.dst[b0] == p.dst[b0 - 1]) begin = p.seg_hi[p.dst[b0]];
    if (b1 < p.m_f && p.dst[b1] == p.dst[b1 - 1]) stop = p.seg_hi[p.dst[b1]];

    u32 cur = NONE;
    // the current segment's role: live at this layer, at its job's last
    // layer, with an end vertex that admits it; its job (PACKED)
    bool seg_live = true, seg_last = last, seg_end_ok = true;
    u32 seg_job = 0, seg_start = p.start;

    auto finish_segment = [&]() {
        if (cur == NONE || !seg_live || !seg_last || !seg_end_ok) return;
        if (PACKED) {
#pragma unroll
            for (int i = 0; i < LPT; i++) {
                const u64 v = gf_mul(xc[i], acc[i]);
                if (v) atomicXor(&p.pout[(u64)seg_job * Lw + lane0 + i], v);
            }
        } else {
#pragma unroll
            for (int i = 0; i < LPT; i++) q[i] ^= gf_mul(xc[i], acc[i]);
        }
    };

    for (u64 base = begin; base < stop; base += T) {
        const u64 e = base + tt;
        u32 s = 0, d = NONE, ci = NONE, co = NONE;
        u64 y = 0;
        if (e < stop) {
            s = p.src[e];
            d = p.dst[e];
            const u32 t = p.time[e];
            if (INNER || p.ell > 2) ci = p.cp_in[e];
            if (PACKED) {
                const PackJob &J = p.pjobs[p.jv[d]];
                if (p.ell < J.k) co = p.cp_out[e];
                if (p.ell <= J.k) y = coef_y(mix64(J.ky ^ (((u64)(s - J.vbase) << 32) | (d - J.vbase))), t, p.ell - 1);
            } else {
                if (INNER || !last) co = p.cp_out[e];
                y = coef_y(mix64(p.ky ^ (((u64)s << 32) | d)), t, p.ell - 1);
            }
        }
        const int cnt = (int)min((u64)T, stop - base);
        for (int j = 0; j < cnt; j++) {
            const u32 dj = __shfl_sync(team_mask, d, j, T);
            const u32 sj = INNER ? 0u : __shfl_sync(team_mask, s, j, T);
            const u32 cij = __shfl_sync(team_mask, ci, j, T);
            const u32 coj = __shfl_sync(team_mask, co, j, T);
            const u64 yj = __shfl_sync(team_mask, y, j, T);
            if (dj != cur) {
                finish_segment();
                cur = dj;
                if (PACKED) {
                    seg_job = p.jv[dj];
                    const PackJob &J = p.pjobs[seg_job];
                    seg_live = p.ell <= J.k;
                    seg_last = p.ell == J.k;
                    seg_end_ok = J.end == NONE || dj == J.end;
                    seg_start = J.start;
                } else {
                    seg_end_ok = p.end == NONE || dj == p.end;
                }
                if constexpr (LPT == 1) {
                    xc[0] = p.x[(u64)dj * Lw + lane0];
                    acc[0] = 0;
                } else {
#pragma unroll
                    for (int i = 0; i < LPT; i += 2) {
                        const ulonglong2 xv = *(const ulonglong2 *)(p.x + (u64)dj * Lw + lane0 + i);
                        xc[i] = xv.x;
                        xc[i + 1] = xv.y;
                        acc[i] = acc[i + 1] = 0;
                    }
                }
            }
            if (PACKED && !seg_live) continue;  // past this job's last layer (uniform in the team)
            const u64 *row = nullptr;
            if (!INNER && p.ell == 2) {
                if (seg_start == NONE || sj == seg_start) row = p.x + (u64)sj * Lw + lane0;
            } else if (cij != NONE) {
                row = p.Cin + (u64)cij * Lw + lane0;
            }
            if (row) {  // uniform across the team
                u64 in[LPT], h[LPT];
                if constexpr (LPT == 1) {
                    in[0] = row[0];
                } else {
#pragma unroll
                    for (int i = 0; i < LPT; i += 2) {
                        const ulonglong2 v = *(const ulonglong2 *)(row + i);
                        in[i] = v.x;
                        in[i + 1] = v.y;
                    }
                }
                if (TAB) {
                    __syncwarp(team_mask);  // earlier lookups are done
                    gf_table_build(tab, yj, tt, T);
                    __syncwarp(team_mask);  // table complete
#pragma unroll
                    for (int i = 0; i < LPT; i++) h[i] = gf_table_mul(tab, in[i]);
                } else {
#pragma unroll
                    for (int i = 0; i < LPT; i++) h[i] = gf_mul(yj, in[i]);
                }
#pragma unroll
                for (int i = 0; i < LPT; i++) acc[i] ^= h[i];
                if (!PACKED && last && p.arc_sum && seg_end_ok) {
                    // this arc's last-layer term, summed over the lanes
                    u64 v = 0;
#pragma unroll
                    for (int i = 0; i < LPT; i++) v ^= gf_mul(xc[i], h[i]);
#pragma unroll
                    for (int o = T / 2; o > 0; o >>= 1) v ^= __shfl_xor_sync(team_mask, v, o, T);
                    // with several lane groups, teams of other lanes add to the same arc
                    if (tt == 0) {
                        if (p.lane_groups > 1) atomicXor(&p.arc_sum[base + j], v);
                        else p.arc_sum[base + j] ^= v;
                    }
                }
            }
            if (coj != NONE) {
                if constexpr (LPT == 1) {
                    p.Cout[(u64)coj * Lw + lane0] = gf_mul(xc[0], acc[0]);
                } else {
#pragma unroll
                    for (int i = 0; i < LPT; i += 2) {
                        ulonglong2 o;
                        o.x = gf_mul(xc[i], acc[i]);
                        o.y = gf_mul(xc[i + 1], acc[i + 1]);
                        *(ulonglong2 *)(p.Cout + (u64)coj * Lw + lane0 + i) = o;
                    }
                }
            }
        }
    }
    finish_segment();
    if (!PACKED && last) {
        if constexpr (LPT == 1) {
            p.partial[chunk * Lw + lane0] = q[0];
        } else {
#pragma unroll
            for (int i = 0; i < LPT; i += 2)
                *(ulonglong2 *)(p.partial + chunk * Lw + lane0 + i) = make_ulonglong2(q[i], q[i + 1]);
        }
    }
}

}  // namespace tmo
