"""Host-side checks of the C-ABI library (no GPU needed): every symbol that
include/*.h declares is exported by libpc2.so, and the host key set-up
(Sec. III-B) agrees with the oracle and with an independent primality test."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(pc2_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2601_14980_b300 import build

    return ctypes.CDLL(build.build())


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) > 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_keygen_primes_and_oracle_agreement(lib):
    import sympy

    from oracle import paillier as O
    from paper_2601_14980_b300 import pc2

    for nbits in (256, 1024, 2048):
        k = pc2.Key.generate(nbits, 11)
        e = k.export()
        assert sympy.isprime(e["p"]) and sympy.isprime(e["q"])
        assert e["p"] < e["q"] and e["p"].bit_length() == e["q"].bit_length() == nbits // 2
        assert (e["p"] * e["q"]).bit_length() == nbits
        ko = O.derive_key(e["p"], e["q"])
        assert (ko.n, ko.lam, ko.mu) == (e["n"], e["lambda"], e["mu"])
    # deterministic in the seed
    assert pc2.Key.generate(512, 3).export() == pc2.Key.generate(512, 3).export()
    assert pc2.Key.generate(512, 3).export()["n"] != pc2.Key.generate(512, 4).export()["n"]


def test_key_from_primes_validation(lib):
    from paper_2601_14980_b300 import pc2, workloads as W

    p, q = W.primes(512, 1)
    k = pc2.Key.from_primes(q, p)               # order normalised to p < q
    assert k.export()["p"] == p
    with pytest.raises(pc2.Pc2Error):
        pc2.Key.from_primes(p, p)                # p == q
    with pytest.raises(pc2.Pc2Error):
        pc2.Key.from_primes(p, q + 2 if q % 3 else q + 4)   # composite (or wrong): rejected
    with pytest.raises(pc2.Pc2Error):
        pc2.Key.from_primes(p, 101)              # unequal sizes
    pub = k.public()
    assert not pub.has_private and pub.export() == {"n": p * q}


def test_strerror_and_tiled_words(lib):
    from paper_2601_14980_b300 import pc2

    assert pc2.tiled_words(0, 64) == 0
    assert pc2.tiled_words(1, 64) == 32 * 64
    assert pc2.tiled_words(33, 8) == 64 * 8
    lib.pc2_strerror.restype = ctypes.c_char_p
    assert lib.pc2_strerror(-3) != lib.pc2_strerror(-4)
