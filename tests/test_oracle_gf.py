"""Pins for the oracle's GF(2^64) arithmetic and random coefficients.

The field is GF(2)[x]/(f), f = x^64 + x^4 + x^3 + x + 1 (Sec. 6.5 leaves b and f
open; b = 64 follows the paper's footnote and experiments).  Every check here
is against mathematics that holds independently of the oracle: an independent
Python polynomial product, field axioms, Fermat/Frobenius identities and
Rabin's irreducibility test.  splitmix64 is pinned to its published outputs.
"""
import random

import pytest

import oracle

F = (1 << 64) | 0b11011
MASK = (1 << 64) - 1


def py_clmul(a, b):
    r = 0
    while b:
        if b & 1:
            r ^= a
        a <<= 1
        b >>= 1
    return r


def py_polymod(a, m):
    dm = m.bit_length() - 1
    while a.bit_length() - 1 >= dm:
        a ^= m << (a.bit_length() - 1 - dm)
    return a


def py_gf_mul(a, b):
    return py_polymod(py_clmul(a, b), F)


def py_gcd(a, b):
    while b:
        a, b = b, py_polymod(a, b)
    return a


def rnd(rng):
    return rng.getrandbits(64)


def test_x64_reduces_to_0x1b(oracle_mod):
    # x^63 * x = x^64 = x^4 + x^3 + x + 1
    assert oracle.gf_mul(1 << 63, 2) == 0x1B
    assert oracle.gf_mul(2, 1 << 63) == 0x1B


def test_matches_independent_polynomial_product(oracle_mod):
    rng = random.Random(11)
    specials = [0, 1, 2, 1 << 63, MASK, 0x1B, 0x8000000000000001]
    pairs = [(a, b) for a in specials for b in specials]
    pairs += [(rnd(rng), rnd(rng)) for _ in range(400)]
    for a, b in pairs:
        assert oracle.gf_mul(a, b) == py_gf_mul(a, b), (hex(a), hex(b))


def test_field_axioms(oracle_mod):
    rng = random.Random(12)
    mul = oracle.gf_mul
    for _ in range(200):
        a, b, c = rnd(rng), rnd(rng), rnd(rng)
        assert mul(a, b) == mul(b, a)
        assert mul(mul(a, b), c) == mul(a, mul(b, c))
        assert mul(a, b ^ c) == mul(a, b) ^ mul(a, c)
        assert mul(a, 1) == a
        assert mul(a, 0) == 0


def test_inverse(oracle_mod):
    rng = random.Random(13)
    assert oracle.gf_inv(1) == 1
    for _ in range(40):
        a = rnd(rng) | 1
        assert oracle.gf_mul(a, oracle.gf_inv(a)) == 1


def test_frobenius(oracle_mod):
    # a^(2^64) = a for every element of GF(2^64).
    rng = random.Random(14)
    for _ in range(20):
        a = rnd(rng)
        s = a
        for _ in range(64):
            s = oracle.gf_mul(s, s)
        assert s == a


def test_modulus_is_irreducible_rabin():
    # Rabin: f of degree 64 is irreducible iff x^(2^64) = x mod f and
    # gcd(x^(2^32) - x, f) = 1 (64's only prime divisor is 2).
    def xpow2(e):
        r = 2
        for _ in range(e):
            r = py_polymod(py_clmul(r, r), F)
        return r
    assert xpow2(64) == 2
    assert py_gcd(F, xpow2(32) ^ 2) == 1


def test_splitmix64_published_outputs(oracle_mod):
    # First outputs of splitmix64 seeded with 1234567 (Vigna's reference code).
    expected = [6457827717110365317, 3203168211198807973, 9817491932198370423,
                4593380528125082431, 16408922859458223821]
    assert [oracle.query_seed(1234567, r) for r in range(5)] == expected
    assert oracle.fmix64(0) == 0


def test_coefficients_distinct_and_order_free(oracle_mod):
    qs = oracle.query_seed(5, 0)
    ys = {oracle.coef_y(qs, a, b, t, p) for a in range(4) for b in range(4) for t in (1, 2, 9) for p in (1, 2, 3)}
    assert len(ys) == 4 * 4 * 3 * 3
    # y of an arc depends on its direction (the reverse arc is another variable)
    assert oracle.coef_y(qs, 1, 2, 5, 1) != oracle.coef_y(qs, 2, 1, 5, 1)
    vs = {oracle.coef_v(qs, u, d) for u in range(50) for d in range(8)}
    ws = {oracle.coef_w(qs, d, j) for d in range(8) for j in range(8)}
    assert len(vs) == 400 and len(ws) == 64


def test_slots_follow_ascending_colours(oracle_mod):
    sb, sc = oracle.slots(6, [5, 2, 5, 7, 2, 2], 8)
    assert list(sc) == [0, 0, 3, 0, 0, 2, 0, 1]
    assert sb[2] == 0 and sb[5] == 3 and sb[7] == 5


@pytest.mark.parametrize("k", [2, 3, 5])
def test_vertex_x_is_sum_over_labels(oracle_mod, k):
    # x_u^A = sum_{j in A} z_{u,j}, z_{u,j} = sum_{d in S_c(u)} v_{u,d} w_{d,j}
    # (eq. motif:1), computed here term by term with the field product.
    ms = [0] * (k - 1) + [1]
    qs = oracle.query_seed(77, 0)
    sb, sc = oracle.slots(k, ms, 2)
    for color, u in ((0, 3), (1, 9)):
        for point in range(1 << k):
            want = 0
            for j in range(k):
                if (point >> j) & 1:
                    for d in range(sb[color], sb[color] + sc[color]):
                        want ^= py_gf_mul(oracle.coef_v(qs, u, d), oracle.coef_w(qs, d, j))
            assert oracle.vertex_x(qs, k, ms, 2, color, u, point) == want


def test_batch_product_matches_scalar(oracle_mod):
    import numpy as np
    rng = np.random.default_rng(3)
    a = rng.integers(0, 2**64, 1000, dtype=np.uint64)
    b = rng.integers(0, 2**64, 1000, dtype=np.uint64)
    out = oracle.gf_mul_batch(a, b)
    for i in range(0, 1000, 37):
        assert int(out[i]) == py_gf_mul(int(a[i]), int(b[i]))
