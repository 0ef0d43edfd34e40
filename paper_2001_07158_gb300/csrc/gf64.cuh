// gf64.cuh -- GF(2^64) arithmetic and counter-based coefficients on sm_103a.
//
// Field: GF(2)[x] / (x^64 + x^4 + x^3 + x + 1), polynomial basis, bit i of a
// 64-bit word is the coefficient of x^i.  Addition is XOR.  The paper fixes
// only the field size (b = 64, Sec. 6.5 and Sec. 8); the modulus is the
// standard pentanomial for this size.
//
// Multiplication (carry-less product then reduction) is built from 32-bit
// integer multiplies: GB300 has no carry-less multiply instruction, so each
// 32x32 carry-less product spreads both operands over four residue classes
// (bits 0 mod 4, 1 mod 4, ...) with three-bit holes between set bits; an
// ordinary integer product of two such spread words counts at most 8 partial
// products per output bit, which stays inside its 4-bit slot, so the parity
// of each slot is the carry-less bit.  This is the "multiplication with
// holes" of T. Pornin's constant-time GHASH for BearSSL (ghash_ctmul,
// described on bearssl.org under constant-time multiplication), restated
// here for 32-bit operands.  Three such products form the 64x64 product by
// Karatsuba.  The table form, gf_table_mul(), serves multipliers shared by
// many sieve lanes.
#pragma once
#include <stdint.h>

namespace tmo {

typedef unsigned long long u64;
typedef unsigned int u32;

// 32 x 32 -> 64 carry-less product.
__device__ __forceinline__ u64 clmul32(u32 a, u32 b)
{
    const u32 m0 = 0x11111111u, m1 = 0x22222222u, m2 = 0x44444444u, m3 = 0x88888888u;
    u32 a0 = a & m0, a1 = a & m1, a2 = a & m2, a3 = a & m3;
    u32 b0 = b & m0, b1 = b & m1, b2 = b & m2, b3 = b & m3;
    u64 c0 = ((u64)a0 * b0) ^ ((u64)a1 * b3) ^ ((u64)a2 * b2) ^ ((u64)a3 * b1);
    u64 c1 = ((u64)a0 * b1) ^ ((u64)a1 * b0) ^ ((u64)a2 * b3) ^ ((u64)a3 * b2);
    u64 c2 = ((u64)a0 * b2) ^ ((u64)a1 * b1) ^ ((u64)a2 * b0) ^ ((u64)a3 * b3);
    u64 c3 = ((u64)a0 * b3) ^ ((u64)a1 * b2) ^ ((u64)a2 * b1) ^ ((u64)a3 * b0);
    return (c0 & 0x1111111111111111ull) | (c1 & 0x2222222222222222ull) |
           (c2 & 0x4444444444444444ull) | (c3 & 0x8888888888888888ull);
}

// Reduce hi * x^64 + lo modulo f.  x^64 = x^4 + x^3 + x + 1, so hi * x^64
// folds to hi ^ hi<<1 ^ hi<<3 ^ hi<<4 plus the <= 4 bits pushed past x^63,
// which fold once more without overflowing.
__device__ __forceinline__ u64 gf_reduce(u64 lo, u64 hi)
{
    u64 over = (hi >> 63) ^ (hi >> 61) ^ (hi >> 60);
    return lo ^ hi ^ (hi << 1) ^ (hi << 3) ^ (hi << 4) ^ over ^ (over << 1) ^ (over << 3) ^ (over << 4);
}

__device__ __forceinline__ u64 gf_mul(u64 a, u64 b)
{
    u32 al = (u32)a, ah = (u32)(a >> 32), bl = (u32)b, bh = (u32)(b >> 32);
    u64 lo = clmul32(al, bl);
    u64 hi = clmul32(ah, bh);
    u64 mid = clmul32(al ^ ah, bl ^ bh) ^ lo ^ hi;
    return gf_reduce(lo ^ (mid << 32), hi ^ (mid >> 32));
}

// a * x^s mod f for 0 <= s < 61 (the bits shifted out are < 2^s, and
// hi * (x^4 + x^3 + x + 1) < 2^(s+4) <= 2^64, so one fold suffices).
// Branch-free for a per-thread s: the clamped funnel shifts take shift
// amounts up to 32, and a second shift by max(s - 32, 0) or max(32 - s, 0)
// covers the rest (s = 0 gives hi = 0).
__device__ __forceinline__ u64 gf_mul_xpow(u64 a, int s)
{
    const u32 a0 = (u32)a, a1 = (u32)(a >> 32);
    const u32 up = (u32)s, dn = 64u - up;                     // a << up, a >> dn
    const u32 up2 = up > 32u ? up - 32u : 0u, dn2 = dn > 32u ? dn - 32u : 0u;
    const u32 r0 = __funnelshift_lc(0u, a0, up);              // (a << s) low word
    const u32 r1 = __funnelshift_lc(0u, __funnelshift_lc(a0, a1, up), up2);
    const u32 h0 = __funnelshift_rc(__funnelshift_rc(a0, a1, dn), 0u, dn2);
    const u32 h1 = __funnelshift_rc(a1, 0u, dn);
    const u64 hi = ((u64)h1 << 32) | h0;
    return (((u64)r1 << 32) | r0) ^ hi ^ (hi << 1) ^ (hi << 3) ^ (hi << 4);
}

// a * x mod f.
__device__ __forceinline__ u64 gf_mul_x(u64 a)
{
    return (a << 1) ^ ((u64)((long long)a >> 63) & 0x1Bull);
}

// ---------------------------------------------------------------------------
// Products by a multiplier y shared by many lanes: a 16 x 16 table
// tab[i][b] = y * b * x^(4i) mod f (i = nibble position, b = nibble value),
// so y * s = XOR_i tab[i][nibble_i(s)] -- 16 shared-memory loads instead of a
// full carry-less product.  A team of `nthreads` threads builds the 256
// entries together (each thread 256/nthreads of them, nthreads in {8,16,32}).
//
// Layout: row i holds 16 entries = 8 chunks of 16 bytes; chunk c of row i is
// stored at chunk position c ^ (i & 7).  Threads write whole chunks, and with
// this swizzle the chunks that one store instruction writes fall in distinct
// bank groups (rows i..i+3 or i..i+7 of neighbouring threads); a lookup of
// entry b in row i reads position b ^ 2(i & 7), still inside the 128-byte row,
// so the 32 lookups of a warp stay free of bank conflicts.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void gf_table_build(u64 *tab, u64 y, int tt, int nthreads)
{
    if (nthreads == 32) {  // half a row (8 entries) per thread
        const int i = tt >> 1, h = tt & 1;
        const u64 b0 = gf_mul_xpow(y, 4 * i);
        const u64 b1 = gf_mul_x(b0), b2 = gf_mul_x(b1);
        const u64 base = h ? gf_mul_x(b2) : 0ull;
        ulonglong2 *row = (ulonglong2 *)(tab + i * 16);
        const int sw = i & 7, c0 = 4 * h;
        row[(c0 + 0) ^ sw] = make_ulonglong2(base, base ^ b0);
        row[(c0 + 1) ^ sw] = make_ulonglong2(base ^ b1, base ^ b1 ^ b0);
        row[(c0 + 2) ^ sw] = make_ulonglong2(base ^ b2, base ^ b2 ^ b0);
        row[(c0 + 3) ^ sw] = make_ulonglong2(base ^ b2 ^ b1, base ^ b2 ^ b1 ^ b0);
        return;
    }
    const int rows = 16 / nthreads;  // whole rows per thread (1 or 2)
    for (int i = tt * rows; i < (tt + 1) * rows; i++) {
        const u64 b0 = gf_mul_xpow(y, 4 * i);
        const u64 b1 = gf_mul_x(b0), b2 = gf_mul_x(b1), b3 = gf_mul_x(b2);
        ulonglong2 *row = (ulonglong2 *)(tab + i * 16);
        const int sw = i & 7;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const u64 base = h ? b3 : 0ull;
            row[(4 * h + 0) ^ sw] = make_ulonglong2(base, base ^ b0);
            row[(4 * h + 1) ^ sw] = make_ulonglong2(base ^ b1, base ^ b1 ^ b0);
            row[(4 * h + 2) ^ sw] = make_ulonglong2(base ^ b2, base ^ b2 ^ b0);
            row[(4 * h + 3) ^ sw] = make_ulonglong2(base ^ b2 ^ b1, base ^ b2 ^ b1 ^ b0);
        }
    }
}

// Lookup side.  The table must start on a 2 KB boundary of shared memory, so
// that its shared address has bits 0..10 clear: the address of entry b of row
// i is then (address | (b' << 3)) + 128 i, where b' = b ^ 2(i & 7) is the
// swizzled column.  XORing s once with 0xECA86420ECA86420 (nibble i of the
// constant is 2(i & 7)) swizzles all sixteen nibbles at once.  Two masked
// shifts per 32-bit half place every nibble, times 8, in a byte of its own
// (even nibbles in one word, odd nibbles in the other); one byte permute per
// lookup then merges that byte with the table address's upper bytes, and the
// row offset rides in the load's immediate.
#define TM_LDS64(out, addr, off) asm volatile("ld.shared.b64 %0, [%1+" #off "];" : "=l"(out) : "r"(addr))

__device__ __forceinline__ u64 gf_table_mul(const u64 *tab, u64 s)
{
    const u32 ta = (u32)__cvta_generic_to_shared(tab);
    const u64 sw = s ^ 0xECA86420ECA86420ull;
    const u32 lo = (u32)sw, hi = (u32)(sw >> 32);
    // byte j of e* / o*: nibble 2j / 2j+1 of the half, times 8
    const u32 el = (lo << 3) & 0x78787878u, ol = (lo >> 1) & 0x78787878u;
    const u32 eh = (hi << 3) & 0x78787878u, oh = (hi >> 1) & 0x78787878u;
    // byte 0 from the nibble word, bytes 1..3 from the table address
#define TM_NIB(w, j) __byte_perm((w), ta, 0x7650u + (j))
    u64 v0, v1, v2, v3, v4, v5, v6, v7, v8, v9, v10, v11, v12, v13, v14, v15;
    TM_LDS64(v0, TM_NIB(el, 0), 0);
    TM_LDS64(v1, TM_NIB(ol, 0), 128);
    TM_LDS64(v2, TM_NIB(el, 1), 256);
    TM_LDS64(v3, TM_NIB(ol, 1), 384);
    TM_LDS64(v4, TM_NIB(el, 2), 512);
    TM_LDS64(v5, TM_NIB(ol, 2), 640);
    TM_LDS64(v6, TM_NIB(el, 3), 768);
    TM_LDS64(v7, TM_NIB(ol, 3), 896);
    TM_LDS64(v8, TM_NIB(eh, 0), 1024);
    TM_LDS64(v9, TM_NIB(oh, 0), 1152);
    TM_LDS64(v10, TM_NIB(eh, 1), 1280);
    TM_LDS64(v11, TM_NIB(oh, 1), 1408);
    TM_LDS64(v12, TM_NIB(eh, 2), 1536);
    TM_LDS64(v13, TM_NIB(oh, 2), 1664);
    TM_LDS64(v14, TM_NIB(eh, 3), 1792);
    TM_LDS64(v15, TM_NIB(oh, 3), 1920);
#undef TM_NIB
    return ((v0 ^ v1 ^ v2) ^ (v3 ^ v4 ^ v5)) ^ ((v6 ^ v7 ^ v8) ^ (v9 ^ v10 ^ v11)) ^ ((v12 ^ v13 ^ v14) ^ v15);
}

// ---------------------------------------------------------------------------
// Counter-based coefficients (splitmix64 output function, Steele/Lea/Flood
// 2014): every sieve variable is a pure function of (query seed, its indices),
// so any arc order, sort or subgraph gives the same values.
// ---------------------------------------------------------------------------
#define TM_GOLDEN 0x9E3779B97F4A7C15ull
#define TM_TAG_V 0x1111111111111111ull
#define TM_TAG_W 0x2222222222222222ull
#define TM_TAG_Y 0x3333333333333333ull
#define TM_PROBE 0xD1B54A32D192ED03ull

__host__ __device__ __forceinline__ u64 mix64(u64 z)
{
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Per-query keys, one per variable family.
struct QueryKeys {
    u64 kv, kw, ky;
};

__host__ __device__ __forceinline__ QueryKeys make_keys(u64 qseed)
{
    QueryKeys k;
    k.kv = mix64(qseed ^ TM_TAG_V);
    k.kw = mix64(qseed ^ TM_TAG_W);
    k.ky = mix64(qseed ^ TM_TAG_Y);
    return k;
}

// v_{u,d} (vertex u, slot d)
__host__ __device__ __forceinline__ u64 coef_v(const QueryKeys &k, u32 u, u32 d)
{
    return mix64(k.kv ^ (((u64)u << 8) | d));
}
// w_{d,j} (slot d, label j)
__host__ __device__ __forceinline__ u64 coef_w(const QueryKeys &k, u32 d, u32 j)
{
    return mix64(k.kw ^ (((u64)d << 8) | j));
}
// Arc part of y: shared by every walk position of arc a -> b.
__host__ __device__ __forceinline__ u64 coef_y_arc(const QueryKeys &k, u32 a, u32 b)
{
    return mix64(k.ky ^ (((u64)a << 32) | b));
}
// y for arc a -> b at time t, walk position p.
__host__ __device__ __forceinline__ u64 coef_y(u64 arc_key, u32 t, u32 p)
{
    return mix64(arc_key ^ (((u64)t << 8) | p));
}

}  // namespace tmo
