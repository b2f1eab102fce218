"""Pins for the oracle's Paillier layer (oracle/paillier.c).

The oracle computes the paper's definitions literally (g^m r^n and
L(c^lambda) mu).  These tests tie it to facts the paper and the mathematics
fix: decryption inverts encryption, the homomorphic identities of
Definitions 1-2, the closed form g^m = 1 + m n for g = n+1, brute force over a
tiny key, the textbook CRT decryption, Lemmas 1-2 (CRT recombination), and the
published Philox test vectors."""
import math
import os
import random

import numpy as np
import pytest

from oracle import paillier as P
from paper_2601_14980_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _key(nbits, seed=1):
    p, q = W.primes(nbits, seed)
    return P.derive_key(p, q)


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert P.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


def test_r_raw_layout():
    # word 4j+i of r_raw is output i of block j, counter (j, e_lo, e_hi, stream)
    seed, stream, e = 0x0123456789ABCDEF, 7, (5 << 32) | 9
    words = 10
    rr = P.r_raw(seed, stream, e, words)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    expect = []
    for j in range(3):
        expect += P.philox4x32_10([j, e & 0xFFFFFFFF, e >> 32, stream], key)
    assert rr == sum(w << (32 * i) for i, w in enumerate(expect[:words]))


def test_derive_key_closed_forms():
    for nbits in (256, 1024):
        k = _key(nbits)
        assert k.n == k.p * k.q and k.n2 == k.n * k.n
        assert k.lam == P.lcm(k.p - 1, k.q - 1)
        # with g = n+1, L(g^lambda mod n^2) = lambda mod n, so mu = lambda^{-1} mod n
        assert k.mu == pow(k.lam, -1, k.n)


def test_tiny_key_brute_force():
    p, q = 11, 13
    k = P.derive_key(p, q, g=None)
    n, n2 = k.n, k.n2
    rs = [r for r in range(1, n) if math.gcd(r, n) == 1][:6]
    for r in rs:
        ms = list(range(n))
        cs = P.encrypt(k, ms, [r] * n)
        for m, c in zip(ms, cs):
            # g^m r^n by repeated multiplication
            acc = 1
            for _ in range(m):
                acc = acc * (n + 1) % n2
            rn = 1
            for _ in range(n):
                rn = rn * r % n2
            assert c == acc * rn % n2
        assert P.decrypt(k, cs) == ms
    # another generator g (any g in Z*_{n^2} with a valid mu)
    k2 = P.derive_key(p, q, g=2)
    cs = P.encrypt(k2, list(range(n)), [rs[1]] * n)
    assert P.decrypt(k2, cs) == list(range(n))


@pytest.mark.parametrize("nbits", [256, 512, 1024])
def test_roundtrip_and_closed_form(nbits):
    k = _key(nbits)
    cnt = 6
    m = W.uniform_below(k.n, cnt, 11) + [0, k.n - 1]
    r = [P.r_of(k, 99, 3, e) for e in range(len(m))]
    c = P.encrypt(k, m, r)
    for mi, ri, ci in zip(m, r, c):
        assert math.gcd(ri, k.n) == 1
        assert ci == (1 + mi * k.n) * pow(ri, k.n, k.n2) % k.n2   # g = n+1 => g^m = 1 + m n
    assert P.decrypt(k, c) == m


def test_homomorphic_identities():
    k = _key(512, seed=2)
    cnt = 5
    a = W.uniform_below(k.n, cnt, 21)
    b = W.uniform_below(k.n, cnt, 22)
    ca = P.encrypt(k, a, [P.r_of(k, 1, 1, e) for e in range(cnt)])
    cb = P.encrypt(k, b, [P.r_of(k, 1, 2, e) for e in range(cnt)])
    # Definition 1
    assert P.decrypt(k, P.hom_add(k, ca, cb)) == [(x + y) % k.n for x, y in zip(a, b)]
    # Definition 2
    ks = [0, 1, 2, 3, (1 << 64) - 1]
    assert P.decrypt(k, P.hom_scal(k, ca, ks)) == [(kk * x) % k.n for kk, x in zip(ks, a)]
    # several groups
    groups = [P.encrypt(k, W.uniform_below(k.n, cnt, 30 + g), [P.r_of(k, 5, g, e) for e in range(cnt)]) for g in range(4)]
    plains = [P.decrypt(k, g) for g in groups]
    assert P.decrypt(k, P.hom_sum(k, groups)) == [sum(col) % k.n for col in zip(*plains)]
    # Eq. (itq2): alpha (+) K (x) s decrypts to alpha + K s (mod n)
    rows, cols = 3, 4
    K = np.array(W.uniform_below(1 << 28, rows * cols, 40), dtype=np.uint64).reshape(rows, cols)
    al = W.uniform_below(1 << 60, rows, 41)
    s = W.uniform_below(1 << 30, cols, 42)
    cal = P.encrypt(k, al, [P.r_of(k, 6, 0, e) for e in range(rows)])
    cs = P.encrypt(k, s, [P.r_of(k, 6, 1, e) for e in range(cols)])
    out = P.decrypt(k, P.hom_matvec(k, cal, cs, K))
    assert out == [(al[i] + sum(int(K[i, j]) * s[j] for j in range(cols))) % k.n for i in range(rows)]


def test_textbook_crt_decryption_equals_lambda_decryption():
    # Paillier's CRT decryption: m_p = L_p(c^{p-1} mod p^2) h_p mod p,
    # h_p = L_p(g^{p-1} mod p^2)^{-1} mod p, then CRT to mod n.  Computed here
    # with Python integers; must equal the oracle's L(c^lambda) mu mod n.
    k = _key(512, seed=3)
    p, q, n = k.p, k.q, k.n
    g = n + 1
    m = W.uniform_below(n, 6, 50)
    c = P.encrypt(k, m, [P.r_of(k, 2, 9, e) for e in range(6)])
    dec = P.decrypt(k, c)

    def half(ci, pr):
        hp = pow((pow(g, pr - 1, pr * pr) - 1) // pr, -1, pr)
        assert hp == pow(-(n // pr) % pr, -1, pr)     # with g = n+1, h_p = (-q)^{-1} mod p
        return (pow(ci, pr - 1, pr * pr) - 1) // pr * hp % pr

    for ci, mi in zip(c, dec):
        mp, mq = half(ci, p), half(ci, q)
        crt = (mp + p * ((mq - mp) * pow(p, -1, q) % q))
        assert crt == mi


def test_crt_lemmas_recombination():
    # Lemmas 1-2 / Eq. (gA-C-B): x mod n^2 = x' + [(x'' - x') (p^2)^{-1} mod q^2] p^2
    k = _key(512, seed=4)
    p2, q2 = k.p ** 2, k.q ** 2
    inv = pow(p2, -1, q2)
    assert (pow(q2, -1, p2) * q2 + inv * p2) % k.n2 == 1   # Lemma 2 (Bezout)
    rng = random.Random(6)
    for _ in range(50):
        x = rng.randrange(k.n2)
        xp, xq = x % p2, x % q2
        assert xp + ((xq - xp) * inv % q2) * p2 == x
    # exponent reduction mod phi(p^2) = p(p-1) used for r^n mod p^2
    r = P.r_of(k, 8, 1, 0)
    assert pow(r, k.n, p2) == pow(r, k.n % (k.p * (k.p - 1)), p2)


def test_r_raw_congruence_identity():
    # (r + t n)^n = r^n (mod n^2): the ciphertext only depends on r mod n,
    # so an unreduced Philox draw gives the same c as r = r_raw mod n.
    k = _key(512, seed=5)
    for e in range(5):
        rr = P.r_raw(77, 4, e, P.r_words(k.nbits))
        assert P.powmod(rr, k.n, k.n2) == P.powmod(rr % k.n, k.n, k.n2)
        assert pow(rr, k.n, k.p ** 2) == pow(rr % k.n, k.n, k.p ** 2)


@pytest.mark.parametrize("nbits", [256, 1024, 2048])
def test_lifted_route_identity(nbits):
    # The encryption kernels compute r^n mod h^2 (h = p, q; h' the other
    # prime) as s^h mod h^2 with s = (r mod h)^(h' mod (h-1)) mod h: since
    # h | n, r^n mod h^2 depends on r mod h only, and r^h mod h^2 is the
    # (h-1)-th root of unity mod h^2 congruent to r mod h.  Checked against the
    # definition on raw draws wider than n, on r = 0 mod h and on r = 1.
    k = _key(nbits, seed=9)
    rng = random.Random(nbits)
    for h, ho in ((k.p, k.q), (k.q, k.p)):
        h2 = h * h
        draws = [P.r_raw(31, 2, e, P.r_words(k.nbits)) for e in range(6)] + [h * 5, 1, k.n - 1]
        draws += [rng.randrange(1, k.n) for _ in range(6)]
        for rr in draws:
            s = pow(rr % h, ho % (h - 1), h)
            lifted = pow(s, h, h2)
            assert lifted == pow(rr % k.n, k.n, h2)
            assert pow(lifted, h - 1, h2) == (0 if rr % h == 0 else 1)   # a root of unity of order | h-1
            assert lifted % h == pow(rr % h, k.n, h)                        # congruent to r^n mod h
    # the encryption it feeds agrees with the oracle's definition
    r = P.r_of(k, 12, 3, 7)
    cp = pow(pow(r % k.p, k.q % (k.p - 1), k.p), k.p, k.p ** 2) * (1 + 5 * k.n) % (k.p ** 2)
    assert cp == P.encrypt(k, [5], [r])[0] % (k.p ** 2)


def test_hom_scal_wide_pins():
    # Definition 2 with k in Z_n: the oracle's binary exponentiation against
    # Python's pow, the decryption identity D(E(a)^k) = k a mod n, and k = 0, 1.
    k = _key(512, seed=10)
    rng = random.Random(11)
    a = [rng.randrange(k.n) for _ in range(4)]
    c = P.encrypt(k, a, [P.r_of(k, 5, 6, e) for e in range(4)])
    ks = [0, 1, k.n - 1, rng.randrange(k.n)]
    out = P.hom_scal_wide(k, c, ks)
    assert out == [pow(ci, ki, k.n2) for ci, ki in zip(c, ks)]
    assert out[0] == 1 and out[1] == c[1]
    assert P.decrypt(k, out) == [ki * ai % k.n for ai, ki in zip(a, ks)]
