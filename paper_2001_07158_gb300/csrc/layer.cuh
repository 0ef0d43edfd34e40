// layer.cuh -- the team body of the generating-function layer kernel
// (eq. gen-polynomial:3), shared by the per-query kernels (sieve.cu) and the
// packed many-graph batch (pack.cu).
#pragma once
#include "gf64.cuh"
#include "internal.h"

namespace tmo {

// ---------------------------------------------------------------------------
// Staged arc metadata (the STAGED form, warp teams of single-job launches).
// Each team owns two buffers of STAGE_ARCS arcs in shared memory.  Lane 0
// fills a buffer with two 1-D bulk copies (cp.async.bulk, completion counted
// in bytes on the buffer's mbarrier): the arcs' 16-byte records {dst, cp_in,
// cp_out, src} and their times, the latter from the 16-byte boundary at or
// below the first arc.  While the team walks one buffer the copy of the next
// sub-batch lands in the other.  The team then computes every staged arc's y
// once (one arc per thread) into the buffer, and the walk reads an arc's
// fields as two shared-memory broadcasts instead of shuffles.
// ---------------------------------------------------------------------------
constexpr int STAGE_ARCS = 64;
struct StageBuf {
    uint4 rec[STAGE_ARCS];      // {dst, cp_in, cp_out, src}
    u32 time[STAGE_ARCS + 4];   // from the 16-byte boundary at or below the first arc
    u64 y[STAGE_ARCS];          // y_{e, l-1}
};
struct TeamStage {
    StageBuf buf[2];
    u64 bar[2];                 // one mbarrier per buffer
};
static_assert(sizeof(StageBuf) % 16 == 0 && sizeof(TeamStage) % 16 == 0, "bulk copy destinations stay aligned");

// Per-thread view of its team's staging state, carried across the chunks a
// resident team takes.
struct StageState {
    u32 phase = 0;        // bit b: parity of buffer b's next completion
    u32 pending = 0;      // bit b: a copy into buffer b is in flight
    bool broken = false;  // a wait ran out: arcs are read from global memory from now on
};

// A wait on a buffer's mbarrier gives up after this long (ns of the global
// timer), sets TM_STATUS_STAGE_TIMEOUT and the team reads its arcs from
// global memory instead.  The checked build waits 0.1 s, so that its test of
// the timeout path stays short.
#ifdef TMOTIF_CHECKED
constexpr unsigned long long STAGE_WAIT_NS = 100000000ull;
#else
constexpr unsigned long long STAGE_WAIT_NS = 1000000000ull;
#endif

__device__ __forceinline__ u32 smem_u32(const void *p) { return (u32)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void stage_init(TeamStage *ts)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&ts->bar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&ts->bar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Lane 0 of the team: copy arcs [sb, se) (se - sb <= STAGE_ARCS) into buffer b.
// rec is 16 bytes per arc; time is read from index sb & ~3 up to the next
// multiple of 4 at or above se, which the workspace pads.  extra_tx (0 except
// in the checked build's forced-timeout test) is added to the bytes the
// barrier expects, so that the copies land but the wait runs out.
__device__ __forceinline__ void stage_issue(const uint4 *rec, const u32 *time, TeamStage *ts, int b, u64 sb, u64 se,
                                            u32 extra_tx)
{
    StageBuf &B = ts->buf[b];
    const u64 t0 = sb & ~3ull, t1 = (se + 3) & ~3ull;
    const u32 nrec = (u32)(se - sb) * 16u, ntime = (u32)(t1 - t0) * 4u;
    const u32 bar = smem_u32(&ts->bar[b]);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(nrec + ntime + extra_tx)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(B.rec)),
                 "l"((unsigned long long)__cvta_generic_to_global(rec + sb)), "r"(nrec), "r"(bar)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(B.time)),
                 "l"((unsigned long long)__cvta_generic_to_global(time + t0)), "r"(ntime), "r"(bar)
                 : "memory");
}

// Wait for buffer b's completion of the given parity, at most STAGE_WAIT_NS.
__device__ __forceinline__ bool stage_wait(TeamStage *ts, int b, u32 parity)
{
    const u32 bar = smem_u32(&ts->bar[b]);
    unsigned long long t_start = 0;
    for (u32 it = 0;; it++) {
        u32 done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 63u) == 0) {
            const unsigned long long now = global_ns();
            if (it == 0) t_start = now;
            else if (now - t_start > STAGE_WAIT_NS) return false;
        }
    }
}

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
//
// STAGED (warp teams of single-job launches): the arcs' fields come from the
// team's staging buffers (ts, ss) instead of the owner threads' loads and
// shuffles; the arcs, their order and every product are the same.
// ---------------------------------------------------------------------------
template <int T, bool TAB, int LPT, bool PACKED, bool INNER = false, bool STAGED = false>
__device__ __forceinline__ void layer_team(const LayerParams &p, u64 team, u64 *tab, TeamStage *ts = nullptr,
                                           StageState *ss = nullptr)
{
    static_assert(!STAGED || (T == 32 && TAB && !PACKED), "the staged form takes warp teams of one job");
    const int tt = threadIdx.x % T;
    const u32 team_mask = (T == 32) ? 0xffffffffu : (((1u << T) - 1u) << (((threadIdx.x & 31) / T) * T));
    if (team / p.lane_groups >= p.n_chunks) return;
    const u64 chunk = p.order ? p.order[team / p.lane_groups] : team / p.lane_groups;
    const u32 lane0 = (u32)(team % p.lane_groups) * (LPT * T) + LPT * tt;
    if (!TM_IN(lane0 + LPT - 1, p.L, p.status)) return;
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
    if (!TM_IN(stop, p.m_f + 1, p.status)) return;

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

    // one arc (dj <- sj at index e, checkpoints cij / coj, multiplier yj),
    // identical for every lane of the team
    auto arc = [&](u32 dj, u32 sj, u32 cij, u32 coj, u64 yj, u64 e) {
        if (!TM_IN(dj, p.n_vert, p.status) || !TM_IN(e, p.m_f, p.status)) return;
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
        if (PACKED && !seg_live) return;  // past this job's last layer (uniform in the team)
        const u64 *row = nullptr;
        if (!INNER && p.ell == 2) {
            if ((seg_start == NONE || sj == seg_start) && TM_IN(sj, p.n_vert, p.status)) row = p.x + (u64)sj * Lw + lane0;
        } else if (cij != NONE && TM_IN(cij, p.n_cp, p.status)) {
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
                    if (p.lane_groups > 1) atomicXor(&p.arc_sum[e], v);
                    else p.arc_sum[e] ^= v;
                }
            }
        }
        if (coj != NONE && TM_IN(coj, p.n_cp, p.status)) {
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
    };

    if constexpr (STAGED) {
        const u64 nsub = stop > begin ? (stop - begin + STAGE_ARCS - 1) / STAGE_ARCS : 0;
        if (nsub && !ss->broken) {
            if (tt == 0) stage_issue(p.rec, p.time, ts, 0, begin, min(begin + STAGE_ARCS, stop), p.stage_extra_tx);
            ss->pending |= 1u;
        }
        for (u64 b = 0; b < nsub; b++) {
            const int bi = (int)(b & 1);
            const u64 sb = begin + b * STAGE_ARCS, se = min(sb + STAGE_ARCS, stop);
            const int cnt = (int)(se - sb);
            if (b + 1 < nsub && !ss->broken) {  // buffer bi ^ 1 was released at the end of sub-batch b - 1
                if (tt == 0) stage_issue(p.rec, p.time, ts, bi ^ 1, se, min(se + STAGE_ARCS, stop), p.stage_extra_tx);
                ss->pending |= 1u << (bi ^ 1);
            }
            bool staged = false;
            if (!ss->broken) {
                staged = __all_sync(team_mask, stage_wait(ts, bi, (ss->phase >> bi) & 1u));
                if (staged) {
                    ss->phase ^= 1u << bi;
                    ss->pending &= ~(1u << bi);
                } else {
                    ss->broken = true;
                    if (tt == 0 && p.status) atomicOr(p.status, TM_STATUS_STAGE_TIMEOUT);
                }
            }
            if (staged) {
                StageBuf &B = ts->buf[bi];
                const int toff = (int)(sb & 3);
                for (int i = tt; i < cnt; i += T) {
                    const uint4 r = B.rec[i];
                    B.y[i] = coef_y(mix64(p.ky ^ (((u64)r.w << 32) | r.x)), B.time[i + toff], p.ell - 1);
                }
                __syncwarp(team_mask);
                for (int j = 0; j < cnt; j++) {
                    const uint4 r = B.rec[j];
                    arc(r.x, r.w, r.y, (INNER || !last) ? r.z : NONE, B.y[j], sb + j);
                }
                __syncwarp(team_mask);  // buffer bi may be refilled
            } else {  // a copy did not land in time: the same arcs from global memory
                for (int j = 0; j < cnt; j++) {
                    const uint4 r = p.rec[sb + j];
                    arc(r.x, r.w, r.y, (INNER || !last) ? r.z : NONE,
                        coef_y(mix64(p.ky ^ (((u64)r.w << 32) | r.x)), p.time[sb + j], p.ell - 1), sb + j);
                }
            }
        }
    } else {
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
                arc(dj, sj, cij, coj, yj, base + j);
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
