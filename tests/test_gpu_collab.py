"""GPU parity of the collaborative CRT split (Sec. IV-C, Algorithm 3) against
the oracle's steps (oracle/collab.py) and against the one-party entry points:
the edge's masked p^2 halves word for word, the master's ciphertexts equal to
pc2_encrypt and oracle.encrypt, the edge's residues and the master's
decryption equal to pc2_decrypt and the plaintexts."""
import random

import numpy as np
import pytest

from oracle import collab as C
from oracle import paillier as P
from paper_2601_14980_b300 import workloads as W

pytestmark = pytest.mark.gpu

SEED, STREAM = 0xC0, 3


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2601_14980_b300 import pc2

    return torch, pc2, pc2.Context(0)


@pytest.mark.parametrize("nbits,count", [(256, 70), (1024, 45), (2048, 37)])
def test_split_encryption_and_decryption(env, nbits, count):
    torch, pc2, ctx = env
    p, q = W.primes(nbits, 31)
    kg, ko = pc2.Key.from_primes(p, q), P.derive_key(p, q)
    L = kg.limbs
    rng = random.Random(nbits)
    m = W.plaintexts_u64(count, seed=nbits)
    m[0], m[1] = 0, np.uint64(2**64 - 1)
    kap = [0, 2**(32 * L) - 2**64 - 1] + [rng.randrange(2**(32 * L) - 2**64) for _ in range(count - 2)]
    dm = torch.from_numpy(m.view(np.int64)).cuda()
    dk = pc2.ints_to_tiled(ctx, kap, L)
    ow = pc2.collab_mask(ctx, kg, dm, dk, count)
    w = [int(x) for x in m]
    assert pc2.tiled_to_ints(ctx, ow, count, L) == C.mask(ko, w, kap)
    cpm = pc2.collab_edge_encrypt(ctx, kg, ow, count, SEED, STREAM, e0=4)
    r = [P.r_of(ko, SEED, STREAM, 4 + e) for e in range(count)]
    sample = list(range(0, count, 7)) + [count - 1]
    got_cpm = pc2.tiled_to_ints(ctx, cpm, count, L)
    want_cpm = C.edge_encrypt_half(ko, [C.mask(ko, w, kap)[i] for i in sample], [r[i] for i in sample])
    assert [got_cpm[i] for i in sample] == want_cpm
    ct = pc2.collab_master_encrypt(ctx, kg, dm, dk, cpm, count, SEED, STREAM, e0=4)
    ref = pc2.encrypt(ctx, kg, dm, SEED, STREAM, e0=4)
    got = pc2.tiled_to_ints(ctx, ct, count, 2 * L)
    assert got == pc2.tiled_to_ints(ctx, ref, count, 2 * L)
    assert [got[i] for i in sample] == P.encrypt(ko, [w[i] for i in sample], [r[i] for i in sample])
    xp = pc2.collab_edge_reduce(ctx, kg, ct, count)
    assert pc2.tiled_to_ints(ctx, xp, count, L) == C.edge_reduce(ko, got)
    dec = pc2.collab_master_decrypt(ctx, kg, ct, xp, count)
    assert pc2.tiled_to_ints(ctx, dec, count, L) == w
    assert ctx.status() == 0


def test_split_argument_errors(env):
    torch, pc2, ctx = env
    kg = pc2.Key.generate(512, 8)
    buf = torch.zeros(64, dtype=torch.int32, device="cuda")
    with pytest.raises(pc2.Pc2Error):
        pc2.collab_edge_reduce(ctx, kg.public(), buf, 1)
    kb = pc2.Key.generate(3072, 8)
    with pytest.raises(pc2.Pc2Error):
        pc2.collab_edge_reduce(ctx, kb, buf, 1)
