"""Pins for the oracle's plain big-integer layer (oracle/bn.c).

Every check compares against arithmetic the oracle does not use: Python's
built-in integers (multiplication, divmod, three-argument pow) and brute-force
repeated multiplication on tiny moduli."""
import random

import pytest

from oracle import paillier as P


def _rand(rng, words):
    return rng.getrandbits(32 * words)


def test_mul_matches_python():
    rng = random.Random(1)
    for _ in range(300):
        a = _rand(rng, rng.randint(1, 40))
        b = _rand(rng, rng.randint(1, 40))
        assert P.mul(a, b) == a * b
    m = (1 << 2048) - 1
    assert P.mul(m, m) == m * m
    assert P.mul(0, m) == 0


def test_divmod_matches_python_random():
    rng = random.Random(2)
    for _ in range(500):
        u = _rand(rng, rng.randint(1, 60))
        v = _rand(rng, rng.randint(1, 30)) or 1
        assert P.divmod_(u, v) == divmod(u, v)


def test_divmod_structured_words():
    # word patterns that make the quotient estimate of Algorithm D overshoot
    # (and exercise the add-back step): runs of 0, 0x7fffffff, 0x80000000, 0xffffffff
    pats = [0, 1, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFF, 0xFFFFFFFE]
    rng = random.Random(3)
    for _ in range(3000):
        uw = [rng.choice(pats) for _ in range(rng.randint(2, 7))]
        vw = [rng.choice(pats) for _ in range(rng.randint(2, 4))]
        u = sum(w << (32 * i) for i, w in enumerate(uw))
        v = sum(w << (32 * i) for i, w in enumerate(vw)) or 3
        assert P.divmod_(u, v) == divmod(u, v)
    # the classic add-back case, scaled to 32-bit digits
    u = (0x7FFFFFFF << 96) | (0x80000000 << 64)
    v = (0x80000000 << 64) | 1
    assert P.divmod_(u, v) == divmod(u, v)


def test_powmod_matches_python_pow():
    rng = random.Random(4)
    for bits in (64, 256, 1024, 2048):
        for _ in range(6):
            m = rng.getrandbits(bits) | 1
            b = rng.getrandbits(bits + 40)
            e = rng.getrandbits(bits)
            assert P.powmod(b, e, m) == pow(b, e, m)
    # even modulus, exponent 0, modulus 1
    assert P.powmod(12345, 678, 1 << 100) == pow(12345, 678, 1 << 100)
    assert P.powmod(5, 0, 97) == 1
    assert P.powmod(5, 3, 1) == 0


def test_powmod_brute_force_tiny():
    # repeated multiplication, no exponentiation algorithm at all
    for m in (2, 3, 10, 97, 143, 221, 255, 1000):
        for b in range(0, 40, 3):
            acc = 1 % m
            for e in range(0, 60):
                assert P.powmod(b, e, m) == acc, (b, e, m)
                acc = acc * b % m


def test_modinv():
    rng = random.Random(5)
    for _ in range(100):
        m = rng.getrandbits(rng.randint(8, 1024)) | 1
        a = rng.getrandbits(1100)
        try:
            x = P.modinv(a, m)
        except ValueError:
            import math

            assert math.gcd(a, m) != 1
            continue
        assert (a * x) % m == 1 % m
    with pytest.raises(ValueError):
        P.modinv(6, 9)
