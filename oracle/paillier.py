"""Python face of the C oracle (oracle/bn.c, oracle/paillier.c).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Integers cross the boundary as Python ints; the C code does the arithmetic.
Each function names the passage of the paper it follows.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass
from typing import Sequence

import numpy as np

from . import build as _build

_lib = ctypes.CDLL(_build.build())
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def _words(x: int, nw: int) -> np.ndarray:
    if x < 0 or x.bit_length() > 32 * nw:
        raise ValueError("integer does not fit in %d words" % nw)
    return np.frombuffer(x.to_bytes(4 * nw, "little"), dtype=np.uint32).copy()


def _int(w: np.ndarray) -> int:
    return int.from_bytes(np.ascontiguousarray(w, dtype=np.uint32).tobytes(), "little")


def _ptr(a: np.ndarray, ty=_u32p):
    return a.ctypes.data_as(ty)


def nwords(x: int) -> int:
    return max(1, (x.bit_length() + 31) // 32)


# ---------------------------------------------------------------- plain big-int


def powmod(b: int, e: int, m: int) -> int:
    """b^e mod m by left-to-right binary exponentiation (oracle/bn.c)."""
    bl, el, ml = nwords(b), nwords(e), nwords(m)
    out = np.zeros(ml, np.uint32)
    rc = _lib.orc_powmod(_ptr(_words(b, bl)), bl, _ptr(_words(e, el)), el, _ptr(_words(m, ml)), ml, _ptr(out))
    if rc:
        raise ZeroDivisionError("modulus is zero")
    return _int(out)


def mul(a: int, b: int) -> int:
    al, bl = nwords(a), nwords(b)
    out = np.zeros(al + bl, np.uint32)
    _lib.orc_mul(_ptr(_words(a, al)), al, _ptr(_words(b, bl)), bl, _ptr(out))
    return _int(out)


def divmod_(u: int, v: int) -> tuple[int, int]:
    """Knuth Algorithm D (oracle/bn.c)."""
    ul, vl = nwords(u), nwords(v)
    q, r = np.zeros(ul, np.uint32), np.zeros(vl, np.uint32)
    if _lib.orc_divmod(_ptr(_words(u, ul)), ul, _ptr(_words(v, vl)), vl, _ptr(q), _ptr(r)):
        raise ZeroDivisionError
    return _int(q), _int(r)


def modinv(a: int, m: int) -> int:
    al, ml = nwords(a), nwords(m)
    out = np.zeros(ml, np.uint32)
    if _lib.orc_modinv(_ptr(_words(a, al)), al, _ptr(_words(m, ml)), ml, _ptr(out)):
        raise ValueError("not invertible")
    return _int(out)


# ---------------------------------------------------------------- Philox / r


def philox4x32_10(ctr: Sequence[int], key: Sequence[int]) -> list[int]:
    """One Philox4x32-10 block (Salmon et al., SC'11)."""
    c = np.array(ctr, np.uint32)
    k = np.array(key, np.uint32)
    out = np.zeros(4, np.uint32)
    _lib.orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return [int(x) for x in out]


def r_raw(seed: int, stream: int, e: int, words: int) -> int:
    """The counter-based draw behind r in Eq. (itq1): word 4j+i is Philox
    output i for counter (j, e_lo, e_hi, stream), key (seed_lo, seed_hi)."""
    out = np.zeros(words, np.uint32)
    _lib.orc_r_raw(ctypes.c_uint64(seed), ctypes.c_uint32(stream), ctypes.c_uint64(e), words, _ptr(out))
    return _int(out)


def r_words(nbits: int) -> int:
    """Width of r_raw: the modulus width plus 64 bits (bias <= 2^-64)."""
    return (nbits + 31) // 32 + 2


# ---------------------------------------------------------------- Paillier


@dataclass(frozen=True)
class Key:
    """Paillier key from the key-generation list of Sec. III-B."""

    p: int
    q: int
    n: int
    n2: int
    g: int
    lam: int  # epsilon = lcm(p-1, q-1) in the paper's notation
    mu: int
    nbits: int

    @property
    def nw(self) -> int:
        return self.nbits // 32


def derive_key(p: int, q: int, g: int | None = None) -> Key:
    """n = pq, lambda = lcm(p-1,q-1), mu = L(g^lambda mod n^2)^{-1} mod n
    (Sec. III-B; L(x) = (x-1)/n).  g defaults to n+1."""
    pw = max(nwords(p), nwords(q))
    n_bits = (p * q).bit_length()
    nw = (n_bits + 31) // 32
    n_guess = p * q
    g = n_guess + 1 if g is None else g
    outs = [np.zeros(nw, np.uint32), np.zeros(2 * nw, np.uint32), np.zeros(nw, np.uint32), np.zeros(nw, np.uint32)]
    rc = _lib.orc_paillier_derive(
        _ptr(_words(p, pw)), _ptr(_words(q, pw)), pw, _ptr(_words(g, 2 * nw)), 2 * nw, nw, *[_ptr(o) for o in outs]
    )
    if rc:
        raise ValueError("g is not a valid Paillier base")
    n, n2, lam, mu = (_int(o) for o in outs)
    return Key(p=p, q=q, n=n, n2=n2, g=g, lam=lam, mu=mu, nbits=32 * nw)


def r_of(key: Key, seed: int, stream: int, e: int) -> int:
    """r = r_raw mod n for element e (Eq. (itq1)'s r, drawn from Philox)."""
    return r_raw(seed, stream, e, r_words(key.nbits)) % key.n


def encrypt(key: Key, m: Sequence[int], r: Sequence[int]) -> list[int]:
    """Eq. (itq1): c = g^m r^n mod n^2, literally (two exponentiations)."""
    cnt = len(m)
    if cnt == 0:
        return []
    nw = key.nw
    mw = nw
    rw = nw
    ma = np.concatenate([_words(int(x), mw) for x in m])
    ra = np.concatenate([_words(int(x), rw) for x in r])
    out = np.zeros(cnt * 2 * nw, np.uint32)
    _lib.orc_paillier_encrypt(_ptr(_words(key.n, nw)), nw, _ptr(_words(key.g, 2 * nw)), _ptr(ma), mw, _ptr(ra), rw, cnt, _ptr(out))
    return [_int(out[i * 2 * nw:(i + 1) * 2 * nw]) for i in range(cnt)]


def decrypt(key: Key, c: Sequence[int]) -> list[int]:
    """Sec. III-C: m = L(c^lambda mod n^2) mu mod n, literally."""
    cnt = len(c)
    if cnt == 0:
        return []
    nw = key.nw
    ca = np.concatenate([_words(int(x), 2 * nw) for x in c])
    out = np.zeros(cnt * nw, np.uint32)
    _lib.orc_paillier_decrypt(_ptr(_words(key.n, nw)), nw, _ptr(_words(key.lam, nw)), _ptr(_words(key.mu, nw)), _ptr(ca), cnt, _ptr(out))
    return [_int(out[i * nw:(i + 1) * nw]) for i in range(cnt)]


def hom_sum(key: Key, groups: Sequence[Sequence[int]]) -> list[int]:
    """Definition 1 (Eq. (headd)) over several operands: prod_g c_g mod n^2."""
    ng = len(groups)
    cnt = len(groups[0]) if ng else 0
    if cnt == 0:
        return []
    cw = 2 * key.nw
    ca = np.concatenate([_words(int(x), cw) for grp in groups for x in grp])
    out = np.zeros(cnt * cw, np.uint32)
    _lib.orc_hom_sum(_ptr(_words(key.n2, cw)), cw, _ptr(ca), ng, cnt, _ptr(out))
    return [_int(out[i * cw:(i + 1) * cw]) for i in range(cnt)]


def hom_add(key: Key, a: Sequence[int], b: Sequence[int]) -> list[int]:
    """Definition 1: c1 c2 mod n^2."""
    return hom_sum(key, [a, b])


def hom_scal(key: Key, c: Sequence[int], k: Sequence[int]) -> list[int]:
    """Definition 2 (Eq. (hemul)): c^k mod n^2, k < 2^64."""
    cnt = len(c)
    if cnt == 0:
        return []
    cw = 2 * key.nw
    ca = np.concatenate([_words(int(x), cw) for x in c])
    ka = np.array([int(x) for x in k], np.uint64)
    out = np.zeros(cnt * cw, np.uint32)
    _lib.orc_hom_scal(_ptr(_words(key.n2, cw)), cw, _ptr(ca), _ptr(ka, _u64p), cnt, _ptr(out))
    return [_int(out[i * cw:(i + 1) * cw]) for i in range(cnt)]


def hom_scal_wide(key: Key, c: Sequence[int], k: Sequence[int]) -> list[int]:
    """Definition 2 (Eq. (hemul)) with k in Z_n as the definition states it:
    c^k mod n^2 for full-width k, by the oracle's binary exponentiation."""
    return [powmod(int(ci), int(ki), key.n2) for ci, ki in zip(c, k)]


def hom_matvec(key: Key, alpha: Sequence[int], s: Sequence[int], K: np.ndarray) -> list[int]:
    """Eq. (itq2): out_i = alpha_i (+) sum_j K_ij (x) s_j, i.e.
    alpha_i * prod_j s_j^{K_ij} mod n^2 (Definitions 1 and 2, row by row)."""
    rows, cols = K.shape
    if rows == 0:
        return []
    cw = 2 * key.nw
    aa = np.concatenate([_words(int(x), cw) for x in alpha])
    sa = np.concatenate([_words(int(x), cw) for x in s]) if cols else np.zeros(1, np.uint32)
    ka = np.ascontiguousarray(K, dtype=np.uint64)
    out = np.zeros(rows * cw, np.uint32)
    _lib.orc_hom_matvec(_ptr(_words(key.n2, cw)), cw, _ptr(aa), _ptr(sa), _ptr(ka, _u64p), rows, cols, _ptr(out))
    return [_int(out[i * cw:(i + 1) * cw]) for i in range(rows)]


def lcm(a: int, b: int) -> int:
    return a // math.gcd(a, b) * b
