"""Key-owner encryption (Eq. (itq1) through the CRT halves of Sec. IV-A) and
CRT decryption (Sec. III-C) at 2048-bit n with the full-width powers on the
tensor cores (engine PC2_ENGINE_TC), against the oracle bit for bit and
against the integer-pipe path: ragged tiles of 128 elements, 64-bit and
full-width plaintexts, and a launch with more tiles than resident CTAs."""
import concurrent.futures as cf
import os

import numpy as np
import pytest

from oracle import paillier as O
from paper_2601_14980_b300 import workloads as W

pytestmark = pytest.mark.gpu

SEED, STREAM = 0x7C, 5


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2601_14980_b300 import pc2

    ctx = pc2.Context(0)
    p, q = W.primes(2048, 21)
    return torch, pc2, ctx, pc2.Key.from_primes(p, q), O.derive_key(p, q)


def _pool_encrypt(ko, m, e0s, seed, stream):
    m, e0s = [int(x) for x in m], [int(e) for e in e0s]
    workers = max(1, min(32, os.cpu_count() or 1))
    chunks = [c for c in (list(range(i, len(m), workers)) for i in range(workers)) if c]

    def job(ix):
        return ix, O.encrypt(ko, [m[i] for i in ix], [O.r_of(ko, seed, stream, e0s[i]) for i in ix])

    out = [None] * len(m)
    with cf.ThreadPoolExecutor(workers) as ex:
        for ix, cts in ex.map(job, chunks):
            for i, c in zip(ix, cts):
                out[i] = c
    return out


def _engine(pc2, ctx, eng):
    pc2.set_engine(ctx, eng)


def test_encrypt_decrypt_tensor_cores_against_oracle(env):
    torch, pc2, ctx, kg, ko = env
    count = 300                                   # tiles of 128: two full, one ragged
    m = W.plaintexts_u64(count, seed=3)
    m[0], m[1] = 0, np.uint64(2**64 - 1)
    dm = torch.from_numpy(m.view(np.int64)).cuda()
    try:
        _engine(pc2, ctx, pc2.ENGINE_TC)
        ct = pc2.encrypt(ctx, kg, dm, SEED, STREAM, e0=9)
        got = pc2.tiled_to_ints(ctx, ct, count, 128)
        assert got == _pool_encrypt(ko, m, [9 + i for i in range(count)], SEED, STREAM)
        dec = pc2.tiled_to_ints(ctx, pc2.decrypt(ctx, kg, ct, count), count, 64)
        assert dec == [int(x) for x in m]
        # full-width plaintexts in [0, n), encrypted by the oracle, and by the wide entry point
        mw = [0, 1, ko.n - 1] + W.uniform_below(ko.n, 134, 8)
        cw = _pool_encrypt(ko, mw, list(range(len(mw))), 4, 4)
        dcw = pc2.ints_to_tiled(ctx, cw, 128)
        assert pc2.tiled_to_ints(ctx, pc2.decrypt(ctx, kg, dcw, len(mw)), len(mw), 64) == mw
        ctw = pc2.encrypt_wide(ctx, kg, pc2.ints_to_tiled(ctx, mw, 64), len(mw), 4, 4)
        assert pc2.tiled_to_ints(ctx, ctw, len(mw), 128) == cw
    finally:
        _engine(pc2, ctx, -1)
    assert ctx.status() == 0


def test_tensor_cores_equal_integer_pipe_many_tiles(env):
    """2^16 + 37 elements (more tiles than resident CTAs): ciphertexts and
    decryptions word for word equal to the integer-pipe path."""
    torch, pc2, ctx, kg, ko = env
    count = (1 << 16) + 37
    m = W.plaintexts_u64(count, seed=4)
    dm = torch.from_numpy(m.view(np.int64)).cuda()
    outs = {}
    try:
        for eng in (pc2.ENGINE_IMAD, pc2.ENGINE_TC):
            _engine(pc2, ctx, eng)
            ct = pc2.encrypt(ctx, kg, dm, SEED, STREAM)
            dec = pc2.decrypt(ctx, kg, ct, count)
            outs[eng] = (pc2.unpack(ctx, ct, count, 128), pc2.unpack(ctx, dec, count, 64))
    finally:
        _engine(pc2, ctx, -1)
    torch.cuda.synchronize()
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    w = outs[1][1].cpu().numpy().view(np.uint32).reshape(count, 64)
    assert np.array_equal(w[:, 0].astype(np.uint64) | (w[:, 1].astype(np.uint64) << np.uint64(32)), m)
    assert ctx.status() == 0
