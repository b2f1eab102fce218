"""Collaborative CRT encryption and decryption between the master and an
edge node (the paper's Sec. IV-C, Algorithm 3), in plain big-integer steps.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper splits every computation mod n^2 into its halves mod p^2 and
q^2 (Lemmas 1-2): the master computes the q^2 half, edge node k the p^2
half, after the master has sent p^2 and phi(p^2) once.  Its obfuscation
O(.) is not defined; the reading followed here (additive masking):

* exchange 1 (master -> edge): O(w) = w + kappa for each plaintext w of the
  master's vectors, kappa drawn by the master below 2^(32 L) - 2^64 (L words
  of n), so that O(w) fits in L words;
* edge: a = O(w) mod phi(p^2), then its half of Eq. (itq1),
  c'_masked = g^a r^(n mod phi(p^2)) mod p^2 (Lemma 1's reduced exponents);
* exchange 2 (edge -> master): c'_masked;
* master: c' = c'_masked g^(phi(p^2) - (kappa mod phi(p^2))) mod p^2 (the
  mask removed: g^phi(p^2) = 1 mod p^2), its own half
  c'' = g^(w mod phi(q^2)) r^(n mod phi(q^2)) mod q^2, and Eq. (gA-C-B):
  c = c' + [(c'' - c') (p^2)^-1 mod q^2] p^2, which is E(w; r);
* exchange 3 (master -> edge): the ciphertexts.
Decryption of an edge node's ciphertext x-hat: the edge sends x-hat and
x-hat' = x-hat mod p^2; the master reduces x-hat'' = x-hat mod q^2 itself and
decrypts from the two residues: m_h = L_h(x-hat_h^(h-1) mod h^2) (L_h(g^(h-1)
mod h^2))^-1 mod h for h = p, q, recombined by Garner's rule mod n.

Products, powers, reductions and inverses use the oracle's schoolbook C
routines (oracle/bn.c through oracle.paillier); additions, subtractions and
exact divisions are Python integer operations."""
from __future__ import annotations

from typing import Sequence

from . import paillier as P


def phi_sq(h: int) -> int:
    """phi(h^2) = h (h - 1) for a prime h."""
    return h * (h - 1)


def mask(key: P.Key, w: Sequence[int], kappa: Sequence[int]) -> list[int]:
    """Exchange 1: O(w) = w + kappa (the master's additive mask)."""
    return [int(x) + int(k) for x, k in zip(w, kappa)]


def edge_encrypt_half(key: P.Key, ow: Sequence[int], r: Sequence[int]) -> list[int]:
    """Edge node: a = O(w) mod phi(p^2); c'_masked = g^a r^(n mod phi(p^2)) mod p^2."""
    p2, ph = key.p * key.p, phi_sq(key.p)
    en = P.divmod_(key.n, ph)[1]
    out = []
    for o, ri in zip(ow, r):
        a = P.divmod_(int(o), ph)[1]
        out.append(P.divmod_(P.mul(P.powmod(key.g, a, p2), P.powmod(ri, en, p2)), p2)[1])
    return out


def master_encrypt(key: P.Key, w: Sequence[int], kappa: Sequence[int], cp_masked: Sequence[int],
                   r: Sequence[int]) -> list[int]:
    """Master: unmask the p^2 half, compute the q^2 half, recombine (Eq. (gA-C-B))."""
    p2, q2 = key.p * key.p, key.q * key.q
    php, phq = phi_sq(key.p), phi_sq(key.q)
    enq = P.divmod_(key.n, phq)[1]
    p2inv = P.modinv(P.divmod_(p2, q2)[1], q2)
    out = []
    for wi, ki, cm, ri in zip(w, kappa, cp_masked, r):
        unmask = P.powmod(key.g, php - P.divmod_(int(ki), php)[1], p2)
        c1 = P.divmod_(P.mul(int(cm), unmask), p2)[1]
        c2 = P.divmod_(P.mul(P.powmod(key.g, P.divmod_(int(wi), phq)[1], q2), P.powmod(ri, enq, q2)), q2)[1]
        d = (c2 - c1) % q2
        out.append(c1 + P.divmod_(P.mul(d, p2inv), q2)[1] * p2)
    return out


def edge_reduce(key: P.Key, xhat: Sequence[int]) -> list[int]:
    """Edge node: x-hat' = x-hat mod p^2."""
    p2 = key.p * key.p
    return [P.divmod_(int(c), p2)[1] for c in xhat]


def master_decrypt(key: P.Key, xhat: Sequence[int], xp: Sequence[int]) -> list[int]:
    """Master: m from x-hat' (the edge's residue mod p^2) and x-hat mod q^2."""
    p, q = key.p, key.q
    out = []
    for c, cp in zip(xhat, xp):
        halves = []
        for h, res in ((p, int(cp)), (q, P.divmod_(int(c), q * q)[1])):
            h2 = h * h
            u = P.powmod(res, h - 1, h2)
            gh = P.powmod(key.g, h - 1, h2)
            lu, lg = (u - 1) // h, (gh - 1) // h
            halves.append(P.divmod_(P.mul(lu, P.modinv(lg, h)), h)[1])
        mp, mq = halves
        t = P.divmod_(P.mul((mq - mp) % q, P.modinv(p % q, q)), q)[1]
        out.append(mp + p * t)
    return out
