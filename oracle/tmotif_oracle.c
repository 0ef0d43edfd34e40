/*
 * tmotif_oracle.c -- plain, slow CPU oracle for constrained multilinear
 * sieving of temporal path motifs (Thejaswi, Gionis, Lauri, "Finding path
 * motifs in large temporal graphs using algebraic fingerprints").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * GPU library is checked against.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it; the product library never
 * calls it, and it shares no code, header or table with the GPU path.
 *
 * Everything here is written for a reader to check against the paper by eye:
 *   - GF(2^64) arithmetic is the textbook shift-and-add ("Russian peasant")
 *     product with interleaved reduction modulo f(x) = x^64 + x^4 + x^3 + x + 1.
 *   - The generating function follows eq. (gen-polynomial:3) of Sec. 6.4:
 *       P_{u,1,i} = x_u,
 *       P_{u,l,i} = x_u * sum_{v in N_i(u)} y_{uv,l-1,i} P_{v,l-1,i-1} + P_{u,l,i-1}.
 *     or_sieve_points() evaluates it with the time index rolled (one array per
 *     walk length, lengths updated in decreasing order inside each time step so
 *     that P_{.,l-1,i-1} is read before it is overwritten); or_literal_table()
 *     fills the full table P_{u,l,i} exactly as printed, for tiny graphs.
 *   - The sieve variables follow Lemma 6.5 (constrained multilinear sieving,
 *     eq. motif:1): z_{i,j} = sum_{d in S_{c(i)}} v_{i,d} w_{d,j},
 *     z_i^A = sum_{j in A} z_{i,j}; Q = sum_{A subset of L} P_{k,t}(z^A, y).
 *   - or_brute_points() and or_brute_det() evaluate the same sums from the
 *     walk definitions (Sec. 6.3) without the recurrence.
 *   - or_count_paths() is the exhaustive temporal DFS of the experimental
 *     baseline (Sec. 9.1): ground truth for the decision.
 *   - or_extract() is extraction by self-reducibility (Sec. 6.9) with the
 *     halving group test and a temporal DFS on the survivors.
 *
 * Points the paper leaves open are read as follows (the GPU library makes
 * the same readings in code of its own): field modulus x^64+x^4+x^3+x+1;
 * random values from the splitmix64 output function keyed by the query seed
 * and the variable's indices (y by arc content and walk position); slots of
 * the distinct query colours in ascending order; P_{u,1,i} = x_u for i >= 0;
 * arcs directed, undirected edges as two arcs; duplicate arcs merged and
 * self-loops dropped; start/end as restrictions of the first and last
 * vertex; an inclusive time window; extraction candidates in ascending id.
 *
 * Parity pins (tests/test_oracle_*.py): field axioms, x^64 mod f, inverse,
 * Frobenius, Rabin irreducibility, splitmix64 published outputs, the paper's
 * worked example (Fig. tempwalk-encoding-demo), DP == literal table == walk
 * enumeration == determinant identity, cancellation of repeated-vertex walks,
 * decision == exhaustive DFS over many seeds.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef uint64_t u64;
typedef uint32_t u32;
typedef int64_t i64;

#define OR_ANY 0xFFFFFFFFu
#define OR_KMAX 20

/* ------------------------------------------------------------------------ */
/* GF(2^64), polynomial basis, bit i of a word = coefficient of x^i.         */
/* f(x) = x^64 + x^4 + x^3 + x + 1, so x^64 = x^4 + x^3 + x + 1 = 0x1B.      */
/* ------------------------------------------------------------------------ */
u64 or_gf_mul(u64 a, u64 b)
{
    u64 r = 0;
    for (int i = 0; i < 64; i++) {
        if (b & 1u) r ^= a;          /* add a * x^i when bit i of b is set   */
        b >>= 1;
        u64 top = a >> 63;           /* a <- a * x mod f                    */
        a <<= 1;
        if (top) a ^= 0x1Bu;
    }
    return r;
}

/* out[i] = a[i] * b[i] for i < n (the product above, in a loop). */
void or_gf_mul_batch(const u64 *a, const u64 *b, u64 *out, u64 n)
{
    for (u64 i = 0; i < n; i++) out[i] = or_gf_mul(a[i], b[i]);
}

u64 or_gf_pow(u64 a, u64 e)
{
    u64 r = 1;
    while (e) {
        if (e & 1u) r = or_gf_mul(r, a);
        a = or_gf_mul(a, a);
        e >>= 1;
    }
    return r;
}

/* a^(2^64 - 2) is the inverse of a nonzero a (the multiplicative group has
 * order 2^64 - 1); returns 0 for a = 0. */
u64 or_gf_inv(u64 a) { return or_gf_pow(a, 0xFFFFFFFFFFFFFFFEull); }

/* ------------------------------------------------------------------------ */
/* Random coefficients: splitmix64 (Steele, Lea, Flood 2014).                 */
/* ------------------------------------------------------------------------ */
#define OR_GAMMA 0x9E3779B97F4A7C15ull
#define OR_TAG_V 0x1111111111111111ull
#define OR_TAG_W 0x2222222222222222ull
#define OR_TAG_Y 0x3333333333333333ull
#define OR_PROBE 0xD1B54A32D192ED03ull

u64 or_fmix64(u64 z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* r-th output of the splitmix64 generator started from state `seed`. */
u64 or_query_seed(u64 seed, u32 r) { return or_fmix64(seed + (u64)(r + 1) * OR_GAMMA); }

/* seed of the i-th extraction probe (i >= 1). */
u64 or_probe_seed(u64 seed, u32 i) { return or_fmix64(seed ^ ((u64)i * OR_PROBE)); }

/* v_{u,d}: vertex u, slot d (Lemma 6.5). */
u64 or_coef_v(u64 qs, u32 u, u32 d)
{
    return or_fmix64(or_fmix64(qs ^ OR_TAG_V) ^ (((u64)u << 8) | d));
}

/* w_{d,j}: slot d, label j (Lemma 6.5). */
u64 or_coef_w(u64 qs, u32 d, u32 j)
{
    return or_fmix64(or_fmix64(qs ^ OR_TAG_W) ^ (((u64)d << 8) | j));
}

/* y_{ab,p,t}: the arc a->b at time t used at walk position p (Sec. 6.3). */
u64 or_coef_y(u64 qs, u32 a, u32 b, u32 t, u32 p)
{
    u64 h = or_fmix64(or_fmix64(qs ^ OR_TAG_Y) ^ (((u64)a << 32) | b));
    return or_fmix64(h ^ (((u64)t << 8) | p));
}

/* ------------------------------------------------------------------------ */
/* Slots S_s: distinct query colours in ascending order get consecutive      */
/* ranges of mu(s) slots.  slot_begin/slot_count have num_colors entries.    */
/* ------------------------------------------------------------------------ */
int or_slots(u32 k, const u32 *multiset, u32 num_colors, u32 *slot_begin, u32 *slot_count)
{
    for (u32 c = 0; c < num_colors; c++) { slot_begin[c] = 0; slot_count[c] = 0; }
    for (u32 r = 0; r < k; r++) {
        if (multiset[r] >= num_colors) return -1;
        slot_count[multiset[r]]++;
    }
    u32 off = 0;
    for (u32 c = 0; c < num_colors; c++) { slot_begin[c] = off; off += slot_count[c]; }
    return 0;
}

/* W_d^A = sum_{j in A} w_{d,j}, where A = { j : bit j of point }. */
static u64 or_W(u64 qs, u32 d, u32 k, u64 point)
{
    u64 s = 0;
    for (u32 j = 0; j < k; j++)
        if ((point >> j) & 1u) s ^= or_coef_w(qs, d, j);
    return s;
}

/* x_u^A = z_u^A = sum_{j in A} sum_{d in S_{c(u)}} v_{u,d} w_{d,j}
 *       = sum_{d in S_{c(u)}} v_{u,d} W_d^A.  Zero outside the query colours. */
u64 or_vertex_x(u64 qs, u32 k, const u32 *slot_begin, const u32 *slot_count, u32 color, u32 u, u64 point)
{
    u64 s = 0;
    for (u32 d = slot_begin[color]; d < slot_begin[color] + slot_count[color]; d++)
        s ^= or_gf_mul(or_coef_v(qs, u, d), or_W(qs, d, k, point));
    return s;
}

/* ------------------------------------------------------------------------ */
/* Temporal edge set.  E^tau is a set of triples (u,v,j), j >= 1 (Sec. 4):   */
/* undirected edges become two arcs, self-loops are dropped and identical    */
/* arcs are kept once.  Output is sorted by (time, src, dst).                */
/* ------------------------------------------------------------------------ */
typedef struct { u32 t, a, b; } or_arc;

static int or_arc_cmp(const void *x, const void *y)
{
    const or_arc *p = (const or_arc *)x, *q = (const or_arc *)y;
    if (p->t != q->t) return p->t < q->t ? -1 : 1;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    if (p->b != q->b) return p->b < q->b ? -1 : 1;
    return 0;
}

/* Returns the number of canonical arcs (<= 2m), or -1 on invalid input.
 * out_* need room for 2m entries (m if directed). */
i64 or_canon(u32 n, u64 m, const u32 *src, const u32 *dst, const u32 *time, int undirected,
             u32 *out_src, u32 *out_dst, u32 *out_time)
{
    u64 cap = undirected ? 2 * m : m;
    or_arc *arcs = (or_arc *)malloc((cap ? cap : 1) * sizeof(or_arc));
    if (!arcs) return -1;
    u64 c = 0;
    for (u64 e = 0; e < m; e++) {
        if (src[e] >= n || dst[e] >= n || time[e] == 0) { free(arcs); return -1; }
        if (src[e] == dst[e]) continue;
        arcs[c].t = time[e]; arcs[c].a = src[e]; arcs[c].b = dst[e]; c++;
        if (undirected) { arcs[c].t = time[e]; arcs[c].a = dst[e]; arcs[c].b = src[e]; c++; }
    }
    qsort(arcs, c, sizeof(or_arc), or_arc_cmp);
    u64 w = 0;
    for (u64 e = 0; e < c; e++) {
        if (w > 0 && or_arc_cmp(&arcs[w - 1], &arcs[e]) == 0) continue;
        arcs[w++] = arcs[e];
    }
    for (u64 e = 0; e < w; e++) { out_src[e] = arcs[e].a; out_dst[e] = arcs[e].b; out_time[e] = arcs[e].t; }
    free(arcs);
    return (i64)w;
}

/* ------------------------------------------------------------------------ */
/* Query description shared by the sieve routines below.                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    u32 n;            /* vertices                                          */
    u64 m;            /* canonical arcs, sorted by time                     */
    const u32 *src, *dst, *time;
    const u32 *color; /* n entries                                          */
    u32 num_colors;
    const uint8_t *alive; /* n entries or NULL (all alive)                  */
    u32 k;
    const u32 *multiset;  /* k colours                                       */
    u32 start, end;       /* OR_ANY or a vertex                              */
    u32 t_min, t_max;     /* arc used iff t >= t_min and (t_max == 0 or t <= t_max) */
} or_problem;

static int or_check_query(u32 n, const u32 *color, u32 num_colors, u32 k, const u32 *multiset, u32 start,
                          u32 end);

static int or_arc_in_window(const or_problem *P, u32 t)
{
    return t >= P->t_min && (P->t_max == 0 || t <= P->t_max);
}

/* x_u^A for every vertex, at one point (0 for dead vertices and colours
 * outside the query). */
static void or_all_x(const or_problem *P, u64 qs, const u32 *sb, const u32 *sc, u64 point, u64 *x)
{
    for (u32 u = 0; u < P->n; u++) {
        if (P->alive && !P->alive[u]) { x[u] = 0; continue; }
        x[u] = or_vertex_x(qs, P->k, sb, sc, P->color[u], u, point);
    }
}

/* Evaluate Q^A = sum_{u end-ok} P_{u,k,t}(z^A, y) for every point in
 * [p_begin, p_end), time index rolled.  out has p_end - p_begin entries. */
static int or_sieve_core(const or_problem *P, u64 qs, u64 p_begin, u64 p_end, u64 *out)
{
    u32 k = P->k, n = P->n;
    if (k < 2 || k > OR_KMAX) return -1;
    u32 *sb = (u32 *)malloc(sizeof(u32) * (P->num_colors + 1));
    u32 *sc = (u32 *)malloc(sizeof(u32) * (P->num_colors + 1));
    if (or_slots(k, P->multiset, P->num_colors, sb, sc) != 0) { free(sb); free(sc); return -1; }
    int err = 0;
    i64 npts = (i64)(p_end - p_begin);
#pragma omp parallel
    {
        u64 *x = (u64 *)malloc(sizeof(u64) * (n ? n : 1));
        u64 *Pt = (u64 *)malloc(sizeof(u64) * (size_t)(k + 1) * (n ? n : 1)); /* Pt[l*n + u] */
        if (!x || !Pt) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (i64 pi = 0; pi < npts; pi++) {
            if (!x || !Pt) continue;
            u64 point = p_begin + (u64)pi;
            or_all_x(P, qs, sb, sc, point, x);
            memset(Pt, 0, sizeof(u64) * (size_t)(k + 1) * n);
            /* P_{u,1,i} = x_u for every i >= 0 (restricted to the start vertex). */
            for (u32 u = 0; u < n; u++)
                Pt[1 * (size_t)n + u] = (P->start == OR_ANY || P->start == u) ? x[u] : 0;
            /* Walk the time steps i = 1, 2, ... in increasing order.  Entering
             * step i the arrays hold P_{.,l,i-1}; the "+ P_{u,l,i-1}" term of the
             * recurrence is the value already stored. */
            u64 e = 0;
            while (e < P->m) {
                u64 g0 = e;
                u32 i = P->time[e];
                while (e < P->m && P->time[e] == i) e++;
                if (!or_arc_in_window(P, i)) continue;
                for (u32 l = k; l >= 2; l--) {
                    for (u64 a = g0; a < e; a++) {
                        u32 v = P->src[a], u = P->dst[a];   /* arc v -> u at time i */
                        u64 term = or_gf_mul(or_coef_y(qs, v, u, i, l - 1), Pt[(size_t)(l - 1) * n + v]);
                        Pt[(size_t)l * n + u] ^= or_gf_mul(x[u], term);
                    }
                }
            }
            u64 q = 0;
            for (u32 u = 0; u < n; u++)
                if (P->end == OR_ANY || P->end == u) q ^= Pt[(size_t)k * n + u];
            out[pi] = q;
        }
        free(x);
        free(Pt);
    }
    free(sb);
    free(sc);
    return err ? -1 : 0;
}

static void or_fill_problem(or_problem *P, u32 n, u64 m, const u32 *src, const u32 *dst, const u32 *time,
                            const u32 *color, u32 num_colors, const uint8_t *alive, u32 k, const u32 *multiset,
                            u32 start, u32 end, u32 t_min, u32 t_max)
{
    P->n = n; P->m = m; P->src = src; P->dst = dst; P->time = time; P->color = color;
    P->num_colors = num_colors; P->alive = alive; P->k = k; P->multiset = multiset;
    P->start = start; P->end = end; P->t_min = t_min; P->t_max = t_max;
}

/* Public: per-point sieve values over canonical arcs (sorted by time).
 * qseed is the query seed (or_query_seed(seed, r)).  nthreads <= 0: default. */
int or_sieve_points(u32 n, u64 m, const u32 *src, const u32 *dst, const u32 *time, const u32 *color,
                    u32 num_colors, const uint8_t *alive, u32 k, const u32 *multiset, u32 start, u32 end,
                    u32 t_min, u32 t_max, u64 qseed, u64 p_begin, u64 p_end, u64 *out, int nthreads)
{
    or_problem P;
    or_fill_problem(&P, n, m, src, dst, time, color, num_colors, alive, k, multiset, start, end, t_min, t_max);
#ifdef _OPENMP
    int old = omp_get_max_threads();
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    int r = or_sieve_core(&P, qseed, p_begin, p_end, out);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(old);
#endif
    (void)nthreads;
    return r;
}

/* ------------------------------------------------------------------------ */
/* Literal table: P_{u,l,i} for u in [n], l in [1,k], i in [0,T], exactly as */
/* printed in eq. (gen-polynomial:3), loops l > i > u (Sec. 8).  One point.   */
/* table has n*(k+1)*(T+1) entries, index (u*(k+1) + l)*(T+1) + i.           */
/* Returns Q^A = sum_{u end-ok} P_{u,k,T}.                                   */
/* ------------------------------------------------------------------------ */
int or_literal_table(u32 n, u64 m, const u32 *src, const u32 *dst, const u32 *time, const u32 *color,
                     u32 num_colors, const uint8_t *alive, u32 k, const u32 *multiset, u32 start, u32 end,
                     u32 t_min, u32 t_max, u64 qseed, u64 point, u32 T, u64 *table, u64 *q_out)
{
    if (k < 2 || k > OR_KMAX) return -1;
    or_problem P;
    or_fill_problem(&P, n, m, src, dst, time, color, num_colors, alive, k, multiset, start, end, t_min, t_max);
    u32 *sb = (u32 *)malloc(sizeof(u32) * (num_colors + 1));
    u32 *sc = (u32 *)malloc(sizeof(u32) * (num_colors + 1));
    u64 *x = (u64 *)malloc(sizeof(u64) * (n ? n : 1));
    if (or_slots(k, multiset, num_colors, sb, sc) != 0) { free(sb); free(sc); free(x); return -1; }
    or_all_x(&P, qseed, sb, sc, point, x);
#define TAB(u, l, i) table[((size_t)(u) * (k + 1) + (l)) * (T + 1) + (i)]
    memset(table, 0, sizeof(u64) * (size_t)n * (k + 1) * (T + 1));
    for (u32 u = 0; u < n; u++)
        for (u32 i = 0; i <= T; i++)
            TAB(u, 1, i) = (start == OR_ANY || start == u) ? x[u] : 0;
    for (u32 l = 2; l <= k; l++) {
        for (u32 i = 1; i <= T; i++) {
            for (u32 u = 0; u < n; u++) {
                /* x_u * sum over arcs v -> u at time i of y * P_{v,l-1,i-1} */
                u64 s = 0;
                if (or_arc_in_window(&P, i))
                    for (u64 e = 0; e < m; e++)
                        if (time[e] == i && dst[e] == u)
                            s ^= or_gf_mul(or_coef_y(qseed, src[e], u, i, l - 1), TAB(src[e], l - 1, i - 1));
                TAB(u, l, i) = or_gf_mul(x[u], s) ^ TAB(u, l, i - 1);
            }
        }
    }
    u64 q = 0;
    for (u32 u = 0; u < n; u++)
        if (end == OR_ANY || end == u) q ^= TAB(u, k, T);
#undef TAB
    *q_out = q;
    free(sb); free(sc); free(x);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Walk enumeration (Sec. 6.3 definitions, no recurrence).                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    const or_problem *P;
    u64 qs;
    u64 npts;
    const u64 *xs;     /* xs[pt * n + u]: x_u at point pt, when per-point mode */
    u64 *acc;          /* per-point accumulators                              */
    u32 walk[OR_KMAX];
    u32 wt[OR_KMAX];
    /* determinant mode */
    int det_mode;
    const u32 *sb, *sc;
    u64 det_acc;
    u64 nwalks;
    u64 *arc_acc;      /* det mode: per-arc sums of the walks ending with that arc */
} or_enum;

static u64 or_det(u64 *M, u32 k)
{
    /* Gaussian elimination over GF(2^64); char 2 so det = permanent. */
    u64 det = 1;
    for (u32 c = 0; c < k; c++) {
        u32 piv = k;
        for (u32 r = c; r < k; r++) if (M[r * k + c]) { piv = r; break; }
        if (piv == k) return 0;
        if (piv != c)
            for (u32 j = 0; j < k; j++) { u64 t = M[c * k + j]; M[c * k + j] = M[piv * k + j]; M[piv * k + j] = t; }
        det = or_gf_mul(det, M[c * k + c]);
        u64 inv = or_gf_inv(M[c * k + c]);
        for (u32 r = c + 1; r < k; r++) {
            if (!M[r * k + c]) continue;
            u64 f = or_gf_mul(M[r * k + c], inv);
            for (u32 j = c; j < k; j++) M[r * k + j] ^= or_gf_mul(f, M[c * k + j]);
        }
    }
    return det;
}

static void or_walk_done(or_enum *E)
{
    const or_problem *P = E->P;
    u32 k = P->k;
    if (P->end != OR_ANY && E->walk[k - 1] != P->end) return;
    E->nwalks++;
    u64 yprod = 1;
    for (u32 r = 0; r + 1 < k; r++)
        yprod = or_gf_mul(yprod, or_coef_y(E->qs, E->walk[r], E->walk[r + 1], E->wt[r], r + 1));
    if (!E->det_mode) {
        for (u64 pt = 0; pt < E->npts; pt++) {
            u64 mono = yprod;
            for (u32 r = 0; r < k; r++) mono = or_gf_mul(mono, E->xs[pt * P->n + E->walk[r]]);
            E->acc[pt] ^= mono;
        }
    } else {
        /* Z[r][j] = z_{u_r, j} = sum_{d in S_{c(u_r)}} v_{u_r,d} w_{d,j} */
        u64 Z[OR_KMAX * OR_KMAX];
        for (u32 r = 0; r < k; r++) {
            u32 u = E->walk[r];
            int dead = (P->alive && !P->alive[u]);
            u32 c = P->color[u];
            for (u32 j = 0; j < k; j++) {
                u64 z = 0;
                if (!dead)
                    for (u32 d = E->sb[c]; d < E->sb[c] + E->sc[c]; d++)
                        z ^= or_gf_mul(or_coef_v(E->qs, u, d), or_coef_w(E->qs, d, j));
                Z[r * k + j] = z;
            }
        }
        u64 val = or_gf_mul(yprod, or_det(Z, k));
        E->det_acc ^= val;
        if (E->arc_acc) {
            /* the walk's last arc: walk[k-2] -> walk[k-1] at time wt[k-2] */
            for (u64 e = 0; e < P->m; e++)
                if (P->src[e] == E->walk[k - 2] && P->dst[e] == E->walk[k - 1] && P->time[e] == E->wt[k - 2]) {
                    E->arc_acc[e] ^= val;
                    break;
                }
        }
    }
}

static void or_walk_rec(or_enum *E, u32 depth, u32 last_t)
{
    const or_problem *P = E->P;
    if (depth == P->k) { or_walk_done(E); return; }
    u32 cur = E->walk[depth - 1];
    for (u64 e = 0; e < P->m; e++) {
        if (P->src[e] != cur) continue;
        u32 t = P->time[e];
        if (t <= last_t || !or_arc_in_window(P, t)) continue;
        E->walk[depth] = P->dst[e];
        E->wt[depth - 1] = t;
        or_walk_rec(E, depth + 1, t);
    }
}

static void or_walk_all(or_enum *E)
{
    const or_problem *P = E->P;
    for (u32 u = 0; u < P->n; u++) {
        if (P->start != OR_ANY && P->start != u) continue;
        E->walk[0] = u;
        or_walk_rec(E, 1, 0);
    }
}

/* Per-point values by summing every temporal walk's monomial
 * x_{u_1} y_1 x_{u_2} ... y_{k-1} x_{u_k} at the point (Sec. 6.3-6.4).
 * Exponential: tiny graphs only.  Returns the number of walks, -1 on error. */
i64 or_brute_points(u32 n, u64 m, const u32 *src, const u32 *dst, const u32 *time, const u32 *color,
                    u32 num_colors, const uint8_t *alive, u32 k, const u32 *multiset, u32 start, u32 end,
                    u32 t_min, u32 t_max, u64 qseed, u64 p_begin, u64 p_end, u64 *out)
{
    if (k < 2 || k > OR_KMAX) return -1;
    or_problem P;
    or_fill_problem(&P, n, m, src, dst, time, color, num_colors, alive, k, multiset, start, end, t_min, t_max);
    u32 *sb = (u32 *)malloc(sizeof(u32) * (num_colors + 1));
    u32 *sc = (u32 *)malloc(sizeof(u32) * (num_colors + 1));
    if (or_slots(k, multiset, num_colors, sb, sc) != 0) { free(sb); free(sc); return -1; }
    u64 npts = p_end - p_begin;
    u64 *xs = (u64 *)malloc(sizeof(u64) * (size_t)npts * (n ? n : 1));
    for (u64 pt = 0; pt < npts; pt++) or_all_x(&P, qseed, sb, sc, p_begin + pt, xs + pt * n);
    memset(out, 0, sizeof(u64) * npts);
    or_enum E;
    memset(&E, 0, sizeof(E));
    E.P = &P; E.qs = qseed; E.npts = npts; E.xs = xs; E.acc = out; E.det_mode = 0;
    or_walk_all(&E);
    free(xs); free(sb); free(sc);
    return (i64)E.nwalks;
}

/* Whole-sieve value Q = sum over all 2^k points, from the identity
 * sum_{A subset of L} prod_r z_{u_r}^A = det(Z) in characteristic 2, where
 * Z[r][j] = z_{u_r,j} (Lemmas 6.3 and 6.5): Q = sum_walks (prod y) det(Z_walk).
 * Returns the number of walks, -1 on error. */
i64 or_brute_det(u32 n, u64 m, const u32 *src, const u32 *dst, const u32 *time, const u32 *color,
                 u32 num_colors, const uint8_t *alive, u32 k, const u32 *multiset, u32 start, u32 end,
                 u32 t_min, u32 t_max, u64 qseed, u64 *q_out)
{
    if (k < 2 || k > OR_KMAX) return -1;
    or_problem P;
    or_fill_problem(&P, n, m, src, dst, time, color, num_colors, alive, k, multiset, start, end, t_min, t_max);
    u32 *sb = (u32 *)malloc(sizeof(u32) * (num_colors + 1));
    u32 *sc = (u32 *)malloc(sizeof(u32) * (num_colors + 1));
    if (or_slots(k, multiset, num_colors, sb, sc) != 0) { free(sb); free(sc); return -1; }
    or_enum E;
    memset(&E, 0, sizeof(E));
    E.P = &P; E.qs = qseed; E.det_mode = 1; E.sb = sb; E.sc = sc;
    or_walk_all(&E);
    *q_out = E.det_acc;
    free(sb); free(sc);
    return (i64)E.nwalks;
}

/* Per-arc whole-sieve values from the determinant identity: for every arc e,
 * the sum over temporal walks whose last arc is e of (prod y) det(Z_walk).
 * arc_out has m entries (arcs as given).  Returns the number of walks. */
i64 or_brute_arc_det(u32 n, u64 m, const u32 *src, const u32 *dst, const u32 *time, const u32 *color,
                     u32 num_colors, const uint8_t *alive, u32 k, const u32 *multiset, u32 start, u32 end,
                     u32 t_min, u32 t_max, u64 qseed, u64 *arc_out)
{
    if (k < 2 || k > OR_KMAX) return -1;
    or_problem P;
    or_fill_problem(&P, n, m, src, dst, time, color, num_colors, alive, k, multiset, start, end, t_min, t_max);
    u32 *sb = (u32 *)malloc(sizeof(u32) * (num_colors + 1));
    u32 *sc = (u32 *)malloc(sizeof(u32) * (num_colors + 1));
    if (or_slots(k, multiset, num_colors, sb, sc) != 0) { free(sb); free(sc); return -1; }
    memset(arc_out, 0, sizeof(u64) * m);
    or_enum E;
    memset(&E, 0, sizeof(E));
    E.P = &P; E.qs = qseed; E.det_mode = 1; E.sb = sb; E.sc = sc; E.arc_acc = arc_out;
    or_walk_all(&E);
    free(sb); free(sc);
    return (i64)E.nwalks;
}

/* ------------------------------------------------------------------------ */
/* Arc-localised sieve: for each arc e = (a -> b, t) in the window whose head  */
/* b may end the path, S_e = sum over all 2^k points A of the last-layer term */
/* of eq. (gen-polynomial:3) that e contributes,                             */
/*     x_b^A * y_{ba,k-1,t} * P_{a,k-1,t-1}(z^A),                            */
/* i.e. the sieve of Lemma 6.5 applied to the walks whose last arc is e (the */
/* vertex-localised sieve of Sec. 6.7, split further by the last arc).  The  */
/* sum of S_e over the arcs into b is the vertex-localised value Q_b.        */
/* Arcs must be canonical (sorted by time).  arc_out has m entries.          */
/* ------------------------------------------------------------------------ */
int or_arc_sums(u32 n, u64 m, const u32 *src, const u32 *dst, const u32 *time, const u32 *color, u32 num_colors,
                const uint8_t *alive, u32 k, const u32 *multiset, u32 start, u32 end, u32 t_min, u32 t_max,
                u64 qseed, u64 *arc_out)
{
    if (k < 2 || k > OR_KMAX) return -1;
    or_problem Pb;
    or_fill_problem(&Pb, n, m, src, dst, time, color, num_colors, alive, k, multiset, start, end, t_min, t_max);
    const or_problem *P = &Pb;
    u32 *sb = (u32 *)malloc(sizeof(u32) * (num_colors + 1));
    u32 *sc = (u32 *)malloc(sizeof(u32) * (num_colors + 1));
    if (or_slots(k, multiset, num_colors, sb, sc) != 0) { free(sb); free(sc); return -1; }
    u64 *x = (u64 *)malloc(sizeof(u64) * (n ? n : 1));
    u64 *Pt = (u64 *)malloc(sizeof(u64) * (size_t)(k + 1) * (n ? n : 1));
    memset(arc_out, 0, sizeof(u64) * m);
    for (u64 point = 0; point < ((u64)1 << k); point++) {
        or_all_x(P, qseed, sb, sc, point, x);
        memset(Pt, 0, sizeof(u64) * (size_t)(k + 1) * n);
        for (u32 u = 0; u < n; u++)
            Pt[1 * (size_t)n + u] = (start == OR_ANY || start == u) ? x[u] : 0;
        u64 e = 0;
        while (e < m) {
            u64 g0 = e;
            u32 i = time[e];
            while (e < m && time[e] == i) e++;
            if (!or_arc_in_window(P, i)) continue;
            for (u32 l = k; l >= 2; l--) {
                for (u64 a = g0; a < e; a++) {
                    u32 v = src[a], u = dst[a];
                    u64 term = or_gf_mul(x[u], or_gf_mul(or_coef_y(qseed, v, u, i, l - 1), Pt[(size_t)(l - 1) * n + v]));
                    Pt[(size_t)l * n + u] ^= term;
                    if (l == k && (end == OR_ANY || end == u)) arc_out[a] ^= term;
                }
            }
        }
    }
    free(x); free(Pt); free(sb); free(sc);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Extraction by localisation (Sec. 6.9, second approach, with the sieve     */
/* localised to arcs).  Level 1 runs the arc-localised sieve on the query   */
/* and takes the first arc (a1 -> b1, t1) in (dst, time, src) order whose    */
/* value is nonzero: some matching path ends with it.  Level j >= 2 asks for */
/* a path on the remaining colours ending at a_{j-1} with every time below   */
/* t_{j-1}, the vertices already chosen (after a_{j-1}) masked, and takes    */
/* the first nonzero arc into a_{j-1}.  After k-1 levels the arcs chosen,    */
/* read backwards, are the path.  Level j evaluates with seed                */
/* or_probe_seed(seed, j); with repeats > 1 an arc counts when any repeat is */
/* nonzero.                                                                  */
/* ------------------------------------------------------------------------ */
int or_extract_localized(u32 n, u64 m, const u32 *src, const u32 *dst, const u32 *time, int undirected,
                         const u32 *color, u32 num_colors, u32 k, const u32 *multiset, u32 start, u32 end,
                         u32 t_min, u32 t_max, u64 seed, u32 repeats, u32 *verts, u32 *times, int *found)
{
    if (or_check_query(n, color, num_colors, k, multiset, start, end) != 0 || repeats < 1) return -1;
    u64 cap = (undirected ? 2 * m : m) + 1;
    u32 *cs = (u32 *)malloc(sizeof(u32) * cap), *cd = (u32 *)malloc(sizeof(u32) * cap), *ct = (u32 *)malloc(sizeof(u32) * cap);
    i64 mc = or_canon(n, m, src, dst, time, undirected, cs, cd, ct);
    if (mc < 0) { free(cs); free(cd); free(ct); return -1; }
    u64 *sums = (u64 *)malloc(sizeof(u64) * (size_t)(mc + 1));
    uint8_t *positive = (uint8_t *)malloc((size_t)mc + 1);
    uint8_t *alive = (uint8_t *)malloc(n ? n : 1);
    memset(alive, 1, n ? n : 1);
    u32 ms[OR_KMAX];
    for (u32 r = 0; r < k; r++) ms[r] = multiset[r];
    u32 kk = k, cur_end = end, cur_tmax = t_max;
    int rc = 0;
    *found = 0;
    for (u32 level = 1; kk >= 2; level++) {
        memset(positive, 0, (size_t)mc + 1);
        for (u32 r = 0; r < repeats && rc == 0; r++) {
            if (or_arc_sums(n, (u64)mc, cs, cd, ct, color, num_colors, alive, kk, ms, start, cur_end, t_min,
                            cur_tmax, or_query_seed(or_probe_seed(seed, level), r), sums) != 0) rc = -1;
            for (i64 e = 0; e < mc; e++) if (sums[e]) positive[e] = 1;
        }
        if (rc) break;
        /* first positive arc in (dst, time, src) order */
        i64 best = -1;
        for (i64 e = 0; e < mc; e++) {
            if (!positive[e]) continue;
            if (best < 0 || cd[e] < cd[best] || (cd[e] == cd[best] && (ct[e] < ct[best] ||
                (ct[e] == ct[best] && cs[e] < cs[best])))) best = e;
        }
        if (best < 0) break;                       /* no path (or a false negative) */
        u32 a = cs[best], b = cd[best], t = ct[best];
        if (level == 1) verts[k - 1] = b;
        verts[kk - 2] = a;
        times[kk - 2] = t;
        /* drop b's colour from the multiset; b is no longer available */
        for (u32 r = 0; r < kk; r++)
            if (ms[r] == color[b]) { ms[r] = ms[kk - 1]; break; }
        kk--;
        alive[b] = 0;
        if (kk < 2) { *found = 1; break; }
        if (t <= 1) break;
        cur_end = a;
        cur_tmax = t - 1;
    }
    free(sums); free(positive); free(alive); free(cs); free(cd); free(ct);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Exhaustive temporal DFS (Sec. 9.1 baseline): counts temporal paths whose  */
/* vertex colours equal the multiset (distinct vertices, strictly increasing */
/* times, window, start/end).  Stops after `limit` paths when limit > 0.     */
/* ------------------------------------------------------------------------ */
typedef struct {
    const or_problem *P;
    u32 need[256];       /* remaining multiplicity per colour (colours < 256 here) */
    uint8_t *onpath;
    u64 count, limit;
    u32 min_last;        /* least last-arc time over the paths counted */
    u32 walk[OR_KMAX], wt[OR_KMAX];
    u32 *first_v, *first_t; /* first path found */
} or_dfs;

static int or_dfs_rec(or_dfs *D, u32 depth, u32 last_t)
{
    const or_problem *P = D->P;
    if (depth == P->k) {
        if (P->end != OR_ANY && D->walk[P->k - 1] != P->end) return 0;
        if (D->count == 0 || D->wt[P->k - 2] < D->min_last) D->min_last = D->wt[P->k - 2];
        if (D->count == 0 && D->first_v) {
            for (u32 r = 0; r < P->k; r++) D->first_v[r] = D->walk[r];
            for (u32 r = 0; r + 1 < P->k; r++) D->first_t[r] = D->wt[r];
        }
        D->count++;
        return D->limit && D->count >= D->limit;
    }
    u32 cur = D->walk[depth - 1];
    for (u64 e = 0; e < P->m; e++) {
        if (P->src[e] != cur) continue;
        u32 t = P->time[e], v = P->dst[e];
        if (t <= last_t || !or_arc_in_window(P, t)) continue;
        if (D->onpath[v] || (P->alive && !P->alive[v])) continue;
        u32 c = P->color[v];
        if (c >= 256 || D->need[c] == 0) continue;
        D->need[c]--; D->onpath[v] = 1;
        D->walk[depth] = v; D->wt[depth - 1] = t;
        int stop = or_dfs_rec(D, depth + 1, t);
        D->need[c]++; D->onpath[v] = 0;
        if (stop) return 1;
    }
    return 0;
}

static i64 or_dfs_run(const or_problem *P, u64 limit, u32 *first_v, u32 *first_t)
{
    if (P->k < 1 || P->k > OR_KMAX || P->num_colors > 256) return -1;
    or_dfs D;
    memset(&D, 0, sizeof(D));
    D.P = P; D.limit = limit; D.first_v = first_v; D.first_t = first_t;
    for (u32 r = 0; r < P->k; r++) {
        if (P->multiset[r] >= P->num_colors) return -1;
        D.need[P->multiset[r]]++;
    }
    D.onpath = (uint8_t *)calloc(P->n ? P->n : 1, 1);
    for (u32 u = 0; u < P->n; u++) {
        if (P->start != OR_ANY && P->start != u) continue;
        if (P->alive && !P->alive[u]) continue;
        u32 c = P->color[u];
        if (D.need[c] == 0) continue;
        D.need[c]--; D.onpath[u] = 1; D.walk[0] = u;
        int stop = or_dfs_rec(&D, 1, 0);
        D.need[c]++; D.onpath[u] = 0;
        if (stop) break;
    }
    free(D.onpath);
    return (i64)D.count;
}

/* Arcs must be in (time, src, dst) order for the "first path" to follow the
 * (time, dst) visiting rule; or_canon produces that order. */
i64 or_count_paths(u32 n, u64 m, const u32 *src, const u32 *dst, const u32 *time, const u32 *color,
                   u32 num_colors, const uint8_t *alive, u32 k, const u32 *multiset, u32 start, u32 end,
                   u32 t_min, u32 t_max, u64 limit, u32 *first_v, u32 *first_t)
{
    or_problem P;
    or_fill_problem(&P, n, m, src, dst, time, color, num_colors, alive, k, multiset, start, end, t_min, t_max);
    return or_dfs_run(&P, limit, first_v, first_t);
}

/* Least last-arc time over all matching temporal paths (exhaustive DFS);
 * returns the number of paths (0: *min_last untouched). */
i64 or_min_last_time(u32 n, u64 m, const u32 *src, const u32 *dst, const u32 *time, const u32 *color,
                     u32 num_colors, u32 k, const u32 *multiset, u32 start, u32 end, u32 t_min, u32 t_max,
                     u32 *min_last)
{
    or_problem P;
    or_fill_problem(&P, n, m, src, dst, time, color, num_colors, NULL, k, multiset, start, end, t_min, t_max);
    if (P.k < 2 || P.k > OR_KMAX || P.num_colors > 256) return -1;
    or_dfs D;
    memset(&D, 0, sizeof(D));
    D.P = &P;
    for (u32 r = 0; r < P.k; r++) D.need[P.multiset[r]]++;
    D.onpath = (uint8_t *)calloc(P.n ? P.n : 1, 1);
    for (u32 u = 0; u < P.n; u++) {
        if (P.start != OR_ANY && P.start != u) continue;
        u32 c = P.color[u];
        if (D.need[c] == 0) continue;
        D.need[c]--; D.onpath[u] = 1; D.walk[0] = u;
        or_dfs_rec(&D, 1, 0);
        D.need[c]++; D.onpath[u] = 0;
    }
    free(D.onpath);
    if (D.count) *min_last = D.min_last;
    return (i64)D.count;
}

/* ------------------------------------------------------------------------ */
/* Decision (Lemma 6.5 + Lemma 6.4): for each repeat r, Q_r = sum over all  */
/* 2^k points; found = OR_r (Q_r != 0).  per_point (optional) receives the   */
/* repeat-0 values on [p_begin, p_end) (p_end = 0 means all 2^k points).    */
/* Input is the caller's edge list; canonicalised here.                      */
/* ------------------------------------------------------------------------ */
static int or_decide_canon(const or_problem *P, u64 seed, u32 repeats, u64 p_begin, u64 p_end,
                           int *found, u64 *sieve_sum, u64 *per_point)
{
    if (P->k < 2 || P->k > OR_KMAX || repeats < 1) return -1;
    u64 full = (u64)1 << P->k;
    if (p_end == 0) { p_begin = 0; p_end = full; }
    if (p_begin >= p_end || p_end > full) return -1;
    u64 npts = p_end - p_begin;
    u64 *vals = (u64 *)malloc(sizeof(u64) * npts);
    if (!vals) return -1;
    *found = 0;
    for (u32 r = 0; r < repeats; r++) {
        if (or_sieve_core(P, or_query_seed(seed, r), p_begin, p_end, vals) != 0) { free(vals); return -1; }
        u64 q = 0;
        for (u64 i = 0; i < npts; i++) q ^= vals[i];
        if (r == 0) {
            *sieve_sum = q;
            if (per_point) memcpy(per_point, vals, sizeof(u64) * npts);
        }
        if (q != 0) *found = 1;
    }
    free(vals);
    return 0;
}

static int or_check_query(u32 n, const u32 *color, u32 num_colors, u32 k, const u32 *multiset, u32 start, u32 end)
{
    if (k < 2 || k > OR_KMAX) return -1;
    for (u32 r = 0; r < k; r++) if (multiset[r] >= num_colors) return -1;
    for (u32 u = 0; u < n; u++) if (color[u] >= num_colors) return -1;
    if (start != OR_ANY && start >= n) return -1;
    if (end != OR_ANY && end >= n) return -1;
    return 0;
}

int or_decide(u32 n, u64 m, const u32 *src, const u32 *dst, const u32 *time, int undirected, const u32 *color,
              u32 num_colors, const uint8_t *alive, u32 k, const u32 *multiset, u32 start, u32 end, u32 t_min,
              u32 t_max, u64 seed, u32 repeats, u64 p_begin, u64 p_end, int *found, u64 *sieve_sum,
              u64 *per_point, int nthreads)
{
    if (or_check_query(n, color, num_colors, k, multiset, start, end) != 0) return -1;
    u64 cap = (undirected ? 2 * m : m) + 1;
    u32 *cs = (u32 *)malloc(sizeof(u32) * cap), *cd = (u32 *)malloc(sizeof(u32) * cap), *ct = (u32 *)malloc(sizeof(u32) * cap);
    i64 mc = or_canon(n, m, src, dst, time, undirected, cs, cd, ct);
    int r = -1;
    if (mc >= 0) {
        or_problem P;
        or_fill_problem(&P, n, (u64)mc, cs, cd, ct, color, num_colors, alive, k, multiset, start, end, t_min, t_max);
#ifdef _OPENMP
        int old = omp_get_max_threads();
        if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
        r = or_decide_canon(&P, seed, repeats, p_begin, p_end, found, sieve_sum, per_point);
#ifdef _OPENMP
        if (nthreads > 0) omp_set_num_threads(old);
#endif
    }
    (void)nthreads;
    free(cs); free(cd); free(ct);
    return r;
}

/* ------------------------------------------------------------------------ */
/* Static preprocessing sieve (Sec. 8.1 (ii) with eq. gen-polynomial:1).     */
/* The temporal graph is merged into the static graph                        */
/*   E_s = {(a, b) : some canonical arc a -> b, at any time}.                */
/* A vertex is kept iff it lies on at least one static path whose colours   */
/* are M (first vertex = start and last = end when given).  Per point A:    */
/*   F_1(u) = x_u [u start-ok],                                              */
/*   F_l(u) = x_u sum_{(v,u) in E_s} yf(v->u, l-1) F_{l-1}(v),               */
/*   B_1(u) = [u end-ok],                                                    */
/*   B_l(u) = sum_{(u,w) in E_s} yb(u->w, k-l+1) x_w B_{l-1}(w),             */
/*   Q_u^A  = sum_{r=1..k} F_r(u) B_{k-r+1}(u).                              */
/* F_r(u) encodes the walk prefixes of r vertices that end at u, B_{k-r+1}(u) */
/* the k-r vertices that follow u, so each product term is the monomial of  */
/* a whole walk of k vertices with u at position r; the arc from position p */
/* to p+1 carries yf before u and yb from u on.  Q_u = sum_A Q_u^A is       */
/* non-zero (up to the sieve's one-sided error) iff such a walk is a path   */
/* with colours M (Lemmas 6.2-6.5 applied to each vertex's terms).          */
/*   yf(a->b, p) = mix64(mix64(kf ^ (a<<32 | b)) ^ p), kf = mix64(qs ^ 0x4444..44) */
/*   yb(a->b, p) = mix64(mix64(kb ^ (a<<32 | b)) ^ p), kb = mix64(qs ^ 0x5555..55) */
/* ------------------------------------------------------------------------ */
#define OR_TAG_YF 0x4444444444444444ull
#define OR_TAG_YB 0x5555555555555555ull

static u64 or_static_y(u64 qs, u64 tag, u32 a, u32 b, u32 p)
{
    u64 key = or_fmix64(qs ^ tag);
    return or_fmix64(or_fmix64(key ^ (((u64)a << 32) | b)) ^ (u64)p);
}

static int or_u64_cmp(const void *x, const void *y)
{
    u64 a = *(const u64 *)x, b = *(const u64 *)y;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* Distinct pairs (a << 32 | b) of the canonical arcs, ascending. */
static u64 or_static_pairs(const or_problem *P, u64 *pairs)
{
    for (u64 e = 0; e < P->m; e++) pairs[e] = ((u64)P->src[e] << 32) | P->dst[e];
    qsort(pairs, P->m, sizeof(u64), or_u64_cmp);
    u64 w = 0;
    for (u64 e = 0; e < P->m; e++)
        if (w == 0 || pairs[w - 1] != pairs[e]) pairs[w++] = pairs[e];
    return w;
}

static int or_static_core(const or_problem *P, u64 qs, u64 *Qv)
{
    u32 k = P->k, n = P->n;
    u32 *sb = (u32 *)malloc(sizeof(u32) * (P->num_colors + 1));
    u32 *sc = (u32 *)malloc(sizeof(u32) * (P->num_colors + 1));
    u64 *pairs = (u64 *)malloc(sizeof(u64) * (P->m ? P->m : 1));
    if (!sb || !sc || !pairs || or_slots(k, P->multiset, P->num_colors, sb, sc) != 0) {
        free(sb); free(sc); free(pairs);
        return -1;
    }
    u64 ms = or_static_pairs(P, pairs);
    memset(Qv, 0, sizeof(u64) * n);
    int err = 0;
    i64 npts = (i64)1 << k;
#pragma omp parallel
    {
        u64 *x = (u64 *)malloc(sizeof(u64) * (n ? n : 1));
        u64 *F = (u64 *)malloc(sizeof(u64) * (size_t)(k + 1) * (n ? n : 1)); /* F[l*n + u] */
        u64 *B = (u64 *)malloc(sizeof(u64) * (size_t)(k + 1) * (n ? n : 1)); /* B[l*n + u] */
        u64 *acc = (u64 *)calloc(n ? n : 1, sizeof(u64));
        if (!x || !F || !B || !acc) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (i64 pt = 0; pt < npts; pt++) {
            if (!x || !F || !B || !acc) continue;
            or_all_x(P, qs, sb, sc, (u64)pt, x);
            memset(F, 0, sizeof(u64) * (size_t)(k + 1) * n);
            memset(B, 0, sizeof(u64) * (size_t)(k + 1) * n);
            for (u32 u = 0; u < n; u++) {
                F[1 * (size_t)n + u] = (P->start == OR_ANY || P->start == u) ? x[u] : 0;
                B[1 * (size_t)n + u] = (P->end == OR_ANY || P->end == u) ? 1 : 0;
            }
            for (u32 l = 2; l <= k; l++) {
                for (u64 e = 0; e < ms; e++) {
                    u32 a = (u32)(pairs[e] >> 32), b = (u32)pairs[e];
                    /* forward: arc a -> b enters the l-th vertex b */
                    F[(size_t)l * n + b] ^= or_gf_mul(or_static_y(qs, OR_TAG_YF, a, b, l - 1),
                                                      F[(size_t)(l - 1) * n + a]);
                    /* backward: a at position k-l+1 followed by b */
                    B[(size_t)l * n + a] ^= or_gf_mul(or_static_y(qs, OR_TAG_YB, a, b, k - l + 1),
                                                      or_gf_mul(x[b], B[(size_t)(l - 1) * n + b]));
                }
                for (u32 u = 0; u < n; u++) F[(size_t)l * n + u] = or_gf_mul(x[u], F[(size_t)l * n + u]);
            }
            for (u32 u = 0; u < n; u++) {
                u64 q = 0;
                for (u32 r = 1; r <= k; r++)
                    q ^= or_gf_mul(F[(size_t)r * n + u], B[(size_t)(k - r + 1) * n + u]);
                acc[u] ^= q;
            }
        }
#pragma omp critical
        {
            if (acc)
                for (u32 u = 0; u < n; u++) Qv[u] ^= acc[u];
        }
        free(x); free(F); free(B); free(acc);
    }
    free(sb); free(sc); free(pairs);
    return err ? -1 : 0;
}

/* Public: per-vertex static sums Q_u (n values) from the raw edge list, with */
/* the query seed of repeat 0.                                                */
int or_static_through(u32 n, u64 m, const u32 *src, const u32 *dst, const u32 *time, int undirected,
                      const u32 *color, u32 num_colors, const uint8_t *alive, u32 k, const u32 *multiset,
                      u32 start, u32 end, u64 seed, u64 *Qv, int nthreads)
{
    if (or_check_query(n, color, num_colors, k, multiset, start, end) != 0) return -1;
    u64 cap = (undirected ? 2 * m : m) + 1;
    u32 *cs = (u32 *)malloc(sizeof(u32) * cap), *cd = (u32 *)malloc(sizeof(u32) * cap), *ct = (u32 *)malloc(sizeof(u32) * cap);
    i64 mc = or_canon(n, m, src, dst, time, undirected, cs, cd, ct);
    int r = -1;
    if (mc >= 0) {
        or_problem P;
        or_fill_problem(&P, n, (u64)mc, cs, cd, ct, color, num_colors, alive, k, multiset, start, end, 0, 0);
#ifdef _OPENMP
        int old = omp_get_max_threads();
        if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
        r = or_static_core(&P, or_query_seed(seed, 0), Qv);
#ifdef _OPENMP
        if (nthreads > 0) omp_set_num_threads(old);
#endif
    }
    (void)nthreads;
    free(cs); free(cd); free(ct);
    return r;
}

/* Brute force for the static sums: enumerate every static walk of k        */
/* vertices over E_s (from start, to end when given) and, for each position */
/* r of each walk, add to Q_{w_r} either                                     */
/*   det_mode 0: the sum over all 2^k points of the walk's monomial with the  */
/*               yf / yb split at r, or                                       */
/*   det_mode 1: (product of the split y's) * det(Z_walk), the same sum by   */
/*               the characteristic-2 identity sum_A prod_r z^A = det(Z).     */
/* Exponential: tiny graphs only.  Returns the number of walks.               */
typedef struct {
    const or_problem *P;
    const u64 *pairs;
    u64 ms, qs;
    const u32 *sb, *sc;
    const u64 *xs; /* 2^k points x n */
    int det_mode;
    u32 walk[OR_KMAX];
    u64 nwalks;
    u64 *Qv;
} or_senum;

static void or_static_walk_done(or_senum *E)
{
    const or_problem *P = E->P;
    u32 k = P->k, n = P->n;
    if (P->end != OR_ANY && E->walk[k - 1] != P->end) return;
    E->nwalks++;
    u64 det = 0;
    if (E->det_mode) {
        u64 Z[OR_KMAX * OR_KMAX];
        for (u32 r = 0; r < k; r++) {
            u32 u = E->walk[r], c = P->color[u];
            int dead = (P->alive && !P->alive[u]);
            for (u32 j = 0; j < k; j++) {
                u64 z = 0;
                if (!dead)
                    for (u32 d = E->sb[c]; d < E->sb[c] + E->sc[c]; d++)
                        z ^= or_gf_mul(or_coef_v(E->qs, u, d), or_coef_w(E->qs, d, j));
                Z[r * k + j] = z;
            }
        }
        det = or_det(Z, k);
    }
    for (u32 r = 1; r <= k; r++) { /* u = walk[r-1] at position r */
        u64 yprod = 1;
        for (u32 p = 1; p < k; p++) {
            u64 tag = p < r ? OR_TAG_YF : OR_TAG_YB;
            yprod = or_gf_mul(yprod, or_static_y(E->qs, tag, E->walk[p - 1], E->walk[p], p));
        }
        u64 sum = 0;
        if (E->det_mode) {
            sum = or_gf_mul(yprod, det);
        } else {
            for (u64 pt = 0; pt < ((u64)1 << k); pt++) {
                u64 mono = yprod;
                for (u32 i = 0; i < k; i++) mono = or_gf_mul(mono, E->xs[pt * n + E->walk[i]]);
                sum ^= mono;
            }
        }
        E->Qv[E->walk[r - 1]] ^= sum;
    }
}

static void or_static_walk_rec(or_senum *E, u32 depth)
{
    if (depth == E->P->k) { or_static_walk_done(E); return; }
    u32 cur = E->walk[depth - 1];
    for (u64 e = 0; e < E->ms; e++) {
        if ((u32)(E->pairs[e] >> 32) != cur) continue;
        E->walk[depth] = (u32)E->pairs[e];
        or_static_walk_rec(E, depth + 1);
    }
}

i64 or_static_brute(u32 n, u64 m, const u32 *src, const u32 *dst, const u32 *time, int undirected,
                    const u32 *color, u32 num_colors, const uint8_t *alive, u32 k, const u32 *multiset, u32 start,
                    u32 end, u64 seed, int det_mode, u64 *Qv)
{
    if (or_check_query(n, color, num_colors, k, multiset, start, end) != 0) return -1;
    u64 cap = (undirected ? 2 * m : m) + 1;
    u32 *cs = (u32 *)malloc(sizeof(u32) * cap), *cd = (u32 *)malloc(sizeof(u32) * cap), *ct = (u32 *)malloc(sizeof(u32) * cap);
    i64 mc = or_canon(n, m, src, dst, time, undirected, cs, cd, ct);
    if (mc < 0) { free(cs); free(cd); free(ct); return -1; }
    or_problem P;
    or_fill_problem(&P, n, (u64)mc, cs, cd, ct, color, num_colors, alive, k, multiset, start, end, 0, 0);
    u32 *sb = (u32 *)malloc(sizeof(u32) * (num_colors + 1));
    u32 *sc = (u32 *)malloc(sizeof(u32) * (num_colors + 1));
    u64 *pairs = (u64 *)malloc(sizeof(u64) * (P.m ? P.m : 1));
    or_slots(k, multiset, num_colors, sb, sc);
    u64 qs = or_query_seed(seed, 0);
    u64 npts = (u64)1 << k;
    u64 *xs = (u64 *)malloc(sizeof(u64) * (size_t)npts * (n ? n : 1));
    for (u64 pt = 0; pt < npts; pt++) or_all_x(&P, qs, sb, sc, pt, xs + pt * n);
    or_senum E;
    memset(&E, 0, sizeof(E));
    E.P = &P; E.pairs = pairs; E.ms = or_static_pairs(&P, pairs); E.qs = qs; E.sb = sb; E.sc = sc;
    E.xs = xs; E.det_mode = det_mode; E.Qv = Qv;
    memset(Qv, 0, sizeof(u64) * n);
    for (u32 u = 0; u < n; u++) {
        if (start != OR_ANY && start != u) continue;
        E.walk[0] = u;
        or_static_walk_rec(&E, 1);
    }
    free(xs); free(sb); free(sc); free(pairs); free(cs); free(cd); free(ct);
    return (i64)E.nwalks;
}

/* ------------------------------------------------------------------------ */
/* EC-PathMotif (Sec. 7.3): the path's arc times must equal the tuple        */
/* T = (j_1, ..., j_{k-1}), j_1 < ... < j_{k-1}.  The recurrence there keeps */
/* one value per vertex and walk length, with no "stay" term:               */
/*   P_{u,1} = x_u,                                                          */
/*   P_{u,l} = x_u * sum over arcs (v -> u, j_{l-1}) of                     */
/*             y_{vu,l-1,j_{l-1}} * P_{v,l-1},      l = 2..k,               */
/*   Q^A     = sum_{u end-ok} P_{u,k}.                                       */
/* Two vertex arrays per point (O(n) memory, as the paper states).  Arcs    */
/* outside the window [t_min, t_max] are not used either; start restricts   */
/* P_{.,1}, end the final sum.                                               */
/* ------------------------------------------------------------------------ */
static int or_ec_core(const or_problem *P, const u32 *T, u64 qs, u64 p_begin, u64 p_end, u64 *out)
{
    u32 k = P->k, n = P->n;
    u32 *sb = (u32 *)malloc(sizeof(u32) * (P->num_colors + 1));
    u32 *sc = (u32 *)malloc(sizeof(u32) * (P->num_colors + 1));
    if (or_slots(k, P->multiset, P->num_colors, sb, sc) != 0) { free(sb); free(sc); return -1; }
    int err = 0;
    i64 npts = (i64)(p_end - p_begin);
#pragma omp parallel
    {
        u64 *x = (u64 *)malloc(sizeof(u64) * (n ? n : 1));
        u64 *cur = (u64 *)malloc(sizeof(u64) * (n ? n : 1));
        u64 *nxt = (u64 *)malloc(sizeof(u64) * (n ? n : 1));
        if (!x || !cur || !nxt) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (i64 pi = 0; pi < npts; pi++) {
            if (!x || !cur || !nxt) continue;
            or_all_x(P, qs, sb, sc, p_begin + (u64)pi, x);
            for (u32 u = 0; u < n; u++) cur[u] = (P->start == OR_ANY || P->start == u) ? x[u] : 0;
            for (u32 l = 2; l <= k; l++) {
                u32 j = T[l - 2];
                memset(nxt, 0, sizeof(u64) * n);
                if (or_arc_in_window(P, j))
                    for (u64 e = 0; e < P->m; e++) {
                        if (P->time[e] != j) continue;
                        u32 v = P->src[e], u = P->dst[e];
                        nxt[u] ^= or_gf_mul(or_coef_y(qs, v, u, j, l - 1), cur[v]);
                    }
                for (u32 u = 0; u < n; u++) cur[u] = or_gf_mul(x[u], nxt[u]);
            }
            u64 q = 0;
            for (u32 u = 0; u < n; u++)
                if (P->end == OR_ANY || P->end == u) q ^= cur[u];
            out[pi] = q;
        }
        free(x); free(cur); free(nxt);
    }
    free(sb);
    free(sc);
    return err ? -1 : 0;
}

/* Public EC-PathMotif decision from the raw edge list; T holds k-1 strictly */
/* increasing timestamps >= 1.  Outputs as or_decide.                        */
int or_decide_ec(u32 n, u64 m, const u32 *src, const u32 *dst, const u32 *time, int undirected, const u32 *color,
                 u32 num_colors, const uint8_t *alive, u32 k, const u32 *multiset, u32 start, u32 end, u32 t_min,
                 u32 t_max, const u32 *T, u64 seed, u32 repeats, u64 p_begin, u64 p_end, int *found,
                 u64 *sieve_sum, u64 *per_point, int nthreads)
{
    if (or_check_query(n, color, num_colors, k, multiset, start, end) != 0 || repeats < 1) return -1;
    for (u32 i = 0; i + 1 < k; i++)
        if (T[i] == 0 || (i > 0 && T[i] <= T[i - 1])) return -1;
    u64 full = (u64)1 << k;
    if (p_end == 0) { p_begin = 0; p_end = full; }
    if (p_begin >= p_end || p_end > full) return -1;
    u64 cap = (undirected ? 2 * m : m) + 1;
    u32 *cs = (u32 *)malloc(sizeof(u32) * cap), *cd = (u32 *)malloc(sizeof(u32) * cap), *ct = (u32 *)malloc(sizeof(u32) * cap);
    u64 npts = p_end - p_begin;
    u64 *vals = (u64 *)malloc(sizeof(u64) * npts);
    i64 mc = or_canon(n, m, src, dst, time, undirected, cs, cd, ct);
    int r = -1;
    if (mc >= 0 && vals) {
        or_problem P;
        or_fill_problem(&P, n, (u64)mc, cs, cd, ct, color, num_colors, alive, k, multiset, start, end, t_min, t_max);
#ifdef _OPENMP
        int old = omp_get_max_threads();
        if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
        r = 0;
        *found = 0;
        for (u32 rep = 0; rep < repeats && r == 0; rep++) {
            r = or_ec_core(&P, T, or_query_seed(seed, rep), p_begin, p_end, vals);
            if (r != 0) break;
            u64 q = 0;
            for (u64 i = 0; i < npts; i++) q ^= vals[i];
            if (rep == 0) {
                *sieve_sum = q;
                if (per_point) memcpy(per_point, vals, sizeof(u64) * npts);
            }
            if (q != 0) *found = 1;
        }
#ifdef _OPENMP
        if (nthreads > 0) omp_set_num_threads(old);
#endif
    }
    (void)nthreads;
    free(cs); free(cd); free(ct); free(vals);
    return r;
}

/* ------------------------------------------------------------------------ */
/* Optimum timestamp (Sec. 6.8): the least t' for which the query restricted */
/* to arcs with times in [t_min, t'] is YES, by binary search over t' with   */
/* O(log t) decisions (each with the query's seed and repeats):             */
/* lo = max(t_min, 1), hi = t_max (or the largest time); if hi is NO there   */
/* is no path; otherwise while lo < hi: mid = lo + (hi - lo) / 2, YES at mid */
/* sets hi = mid, NO sets lo = mid + 1.                                      */
/* ------------------------------------------------------------------------ */
int or_optimum_time(u32 n, u64 m, const u32 *src, const u32 *dst, const u32 *time, int undirected,
                    const u32 *color, u32 num_colors, u32 k, const u32 *multiset, u32 start, u32 end, u32 t_min,
                    u32 t_max, u64 seed, u32 repeats, u32 *t_opt, int *found, int nthreads)
{
    if (or_check_query(n, color, num_colors, k, multiset, start, end) != 0 || repeats < 1) return -1;
    u64 cap = (undirected ? 2 * m : m) + 1;
    u32 *cs = (u32 *)malloc(sizeof(u32) * cap), *cd = (u32 *)malloc(sizeof(u32) * cap), *ct = (u32 *)malloc(sizeof(u32) * cap);
    i64 mc = or_canon(n, m, src, dst, time, undirected, cs, cd, ct);
    if (mc < 0) { free(cs); free(cd); free(ct); return -1; }
#ifdef _OPENMP
    int old = omp_get_max_threads();
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    (void)nthreads;
    u32 tmax_all = 0;
    for (i64 e = 0; e < mc; e++) if (ct[e] > tmax_all) tmax_all = ct[e];
    u32 lo = t_min > 1 ? t_min : 1, hi = t_max ? t_max : tmax_all;
    int rc = 0, yes = 0;
    u64 q = 0;
    *found = 0;
    *t_opt = 0;
    or_problem P;
    or_fill_problem(&P, n, (u64)mc, cs, cd, ct, color, num_colors, NULL, k, multiset, start, end, t_min, hi);
    if (hi >= lo && mc > 0) {
        if (or_decide_canon(&P, seed, repeats, 0, 0, &yes, &q, NULL) != 0) rc = -1;
        if (rc == 0 && yes) {
            while (lo < hi) {
                u32 mid = lo + (hi - lo) / 2;
                P.t_max = mid;
                if (or_decide_canon(&P, seed, repeats, 0, 0, &yes, &q, NULL) != 0) { rc = -1; break; }
                if (yes) hi = mid;
                else lo = mid + 1;
            }
            if (rc == 0) { *found = 1; *t_opt = lo; }
        }
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(old);
#endif
    free(cs); free(cd); free(ct);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Extraction by self-reducibility (Sec. 6.9): candidates R = vertices whose */
/* colour is in the multiset, ascending id.  shrink(block): if the block is  */
/* not all that is left and the problem with the block removed is still YES */
/* (probe i uses seed or_probe_seed(seed, i)), the block is removed; else a  */
/* block of more than one candidate is halved and both halves are tried in   */
/* order.  The survivors then go to the temporal DFS, which visits start     */
/* vertices in ascending id and arcs in (time, dst) order.                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    or_problem *P;
    uint8_t *alive;
    const u32 *R;
    u64 seed;
    u32 repeats;
    u32 probes;
    u64 n_alive;
    int err;
} or_shrink_state;

static void or_shrink(or_shrink_state *S, u64 lo, u64 hi)
{
    if (S->err) return;
    u64 cnt = 0;
    for (u64 i = lo; i < hi; i++) cnt += S->alive[S->R[i]];
    if (cnt == 0) return;
    if (cnt < S->n_alive) {
        for (u64 i = lo; i < hi; i++) S->alive[S->R[i]] = 0;
        S->probes++;
        int found = 0;
        u64 q = 0;
        if (or_decide_canon(S->P, or_probe_seed(S->seed, S->probes), S->repeats, 0, 0, &found, &q, NULL) != 0) {
            S->err = 1;
            return;
        }
        if (found) { S->n_alive -= cnt; return; }
        /* A block is probed before any of its sub-blocks and blocks probed
         * earlier are disjoint from it, so every candidate in it was alive. */
        for (u64 i = lo; i < hi; i++) S->alive[S->R[i]] = 1;
    }
    if (hi - lo == 1) return;
    u64 mid = lo + (hi - lo) / 2;
    or_shrink(S, lo, mid);
    or_shrink(S, mid, hi);
}

int or_extract(u32 n, u64 m, const u32 *src, const u32 *dst, const u32 *time, int undirected, const u32 *color,
               u32 num_colors, u32 k, const u32 *multiset, u32 start, u32 end, u32 t_min, u32 t_max, u64 seed,
               u32 repeats, u32 *verts, u32 *times, int *found, u32 *n_probes, int nthreads)
{
    if (or_check_query(n, color, num_colors, k, multiset, start, end) != 0 || repeats < 1) return -1;
    u64 cap = (undirected ? 2 * m : m) + 1;
    u32 *cs = (u32 *)malloc(sizeof(u32) * cap), *cd = (u32 *)malloc(sizeof(u32) * cap), *ct = (u32 *)malloc(sizeof(u32) * cap);
    i64 mc = or_canon(n, m, src, dst, time, undirected, cs, cd, ct);
    if (mc < 0) { free(cs); free(cd); free(ct); return -1; }
#ifdef _OPENMP
    int old = omp_get_max_threads();
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    (void)nthreads;
    uint8_t inM[256];
    memset(inM, 0, sizeof(inM));
    for (u32 r = 0; r < k; r++) if (multiset[r] < 256) inM[multiset[r]] = 1;
    uint8_t *alive = (uint8_t *)calloc(n ? n : 1, 1);
    u32 *R = (u32 *)malloc(sizeof(u32) * (n ? n : 1));
    u64 nR = 0;
    for (u32 u = 0; u < n; u++)
        if (color[u] < 256 && inM[color[u]]) { alive[u] = 1; R[nR++] = u; }
    or_problem P;
    or_fill_problem(&P, n, (u64)mc, cs, cd, ct, color, num_colors, alive, k, multiset, start, end, t_min, t_max);
    int rc = 0;
    *found = 0;
    *n_probes = 0;
    int yes = 0;
    u64 q = 0;
    if (or_decide_canon(&P, seed, repeats, 0, 0, &yes, &q, NULL) != 0) rc = -1;
    if (rc == 0 && yes) {
        or_shrink_state S;
        S.P = &P; S.alive = alive; S.R = R; S.seed = seed; S.repeats = repeats; S.probes = 0;
        S.n_alive = nR; S.err = 0;
        or_shrink(&S, 0, nR);
        *n_probes = S.probes;
        if (S.err) rc = -1;
        else {
            i64 c = or_dfs_run(&P, 1, verts, times);
            if (c > 0) *found = 1;
        }
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(old);
#endif
    free(alive); free(R); free(cs); free(cd); free(ct);
    return rc;
}
