"""Pins of the collaborative CRT split (Sec. IV-C, Algorithm 3; oracle/collab.py)
against the oracle's literal Paillier (Eq. (itq1), Sec. III-C), which is itself
pinned against Python integers, brute force and the closed form."""
import random

import pytest

from oracle import collab as C
from oracle import paillier as P
from paper_2601_14980_b300 import workloads as W


def _key(nbits, seed, general_g=False):
    p, q = W.primes(nbits, seed)
    if not general_g:
        return P.derive_key(p, q)
    rng = random.Random(seed)
    n2 = (p * q) ** 2
    while True:  # a random base whose order is a multiple of n: L(g^lambda) invertible
        g = rng.randrange(2, n2)
        try:
            return P.derive_key(p, q, g)
        except ValueError:
            continue


@pytest.mark.parametrize("nbits,general_g", [(256, False), (512, False), (512, True), (1024, False)])
def test_split_encryption_equals_encryption(nbits, general_g):
    key = _key(nbits, 3, general_g)
    rng = random.Random(nbits)
    L = key.nw
    w = [0, 1, 2**64 - 1] + [rng.randrange(2**64) for _ in range(6)]   # quantized values: 64 bits
    kappa = [0, 2**(32 * L) - 2**64 - 1] + [rng.randrange(2**(32 * L) - 2**64) for _ in range(len(w) - 2)]
    r = [P.r_of(key, 11, 2, e) for e in range(len(w))]
    ow = C.mask(key, w, kappa)
    assert all(o < 2**(32 * L) for o in ow)
    cpm = C.edge_encrypt_half(key, ow, r)
    got = C.master_encrypt(key, w, kappa, cpm, r)
    assert got == P.encrypt(key, w, r)
    # the mask is what the master removes: unmasking with another kappa breaks it
    bad = C.master_encrypt(key, w, [k + 1 for k in kappa], cpm, r)
    assert all(b != g for b, g in zip(bad, got))
    # with no mask the edge's half is the plain p^2 half of E(w; r)
    p2 = key.p * key.p
    assert C.edge_encrypt_half(key, w, r) == [c % p2 for c in got]


@pytest.mark.parametrize("nbits,general_g", [(256, False), (512, True), (1024, False)])
def test_split_decryption_equals_decryption(nbits, general_g):
    key = _key(nbits, 4, general_g)
    rng = random.Random(nbits + 1)
    m = [0, 1, key.n - 1] + [rng.randrange(key.n) for _ in range(6)]
    c = P.encrypt(key, m, [P.r_of(key, 5, 1, e) for e in range(len(m))])
    xp = C.edge_reduce(key, c)
    assert xp == [x % (key.p * key.p) for x in c]
    assert C.master_decrypt(key, c, xp) == m == P.decrypt(key, c)


def test_split_ciphertexts_aggregate():
    """Ciphertexts from the split encryption keep Definition 1's property."""
    key = _key(512, 6)
    rng = random.Random(9)
    a = [rng.randrange(2**60) for _ in range(4)]
    b = [rng.randrange(2**60) for _ in range(4)]
    kap = [rng.randrange(2**(32 * key.nw) - 2**64) for _ in range(4)]
    ra = [P.r_of(key, 1, 1, e) for e in range(4)]
    rb = [P.r_of(key, 1, 2, e) for e in range(4)]
    ca = C.master_encrypt(key, a, kap, C.edge_encrypt_half(key, C.mask(key, a, kap), ra), ra)
    cb = C.master_encrypt(key, b, kap, C.edge_encrypt_half(key, C.mask(key, b, kap), rb), rb)
    s = P.hom_add(key, ca, cb)
    assert C.master_decrypt(key, s, C.edge_reduce(key, s)) == [x + y for x, y in zip(a, b)]
