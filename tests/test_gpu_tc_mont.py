"""Montgomery squarings with the reduction on the tensor cores (tcgen05.mma,
bf16 digits, exact FP32 column sums) against the oracle and against the
integer-pipe CIOS product, bit for bit.

y = x^(2^k) R^-(2^k - 1) mod N (k Montgomery squarings, R = 2^2048) for N =
p^2 of a 2048-bit key, the modulus of the encryption's and decryption's
64-limb products.  The expected values come from the oracle's plain
powmod, multiply and division."""
import numpy as np
import pytest

from oracle import paillier as O
from paper_2601_14980_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2601_14980_b300 import pc2

    p, _ = W.primes(2048, 17)
    N = p * p
    assert N.bit_length() > 2016 and N.bit_length() <= 2048 and N & 1
    return torch, pc2, pc2.Context(0), N


def _expect(N, xs, k):
    R = 1 << 2048
    rinv = O.modinv(R % N, N)
    f = O.powmod(rinv, (1 << k) - 1, N)
    return [O.divmod_(O.mul(O.powmod(x, 1 << k, N), f), N)[1] for x in xs]


@pytest.mark.parametrize("k", [1, 5, 33])
def test_both_engines_match_the_oracle(env, k):
    torch, pc2, ctx, N = env
    xs = [0, 1, 2, N - 1, N - 2] + W.uniform_below(N, 295, 100 + k)   # three tiles of 128, ragged tail
    dx = pc2.ints_to_tiled(ctx, xs, 64)
    want = _expect(N, xs, k)
    for engine in (pc2.ENGINE_IMAD, pc2.ENGINE_TC):
        y = pc2.mont_sqr(ctx, N, dx, len(xs), k, engine)
        assert pc2.tiled_to_ints(ctx, y, len(xs), 64) == want, engine
    assert ctx.status() == 0


def test_tensor_core_engine_full_grid(env):
    """More tiles than resident CTAs (persistent loop), every element equal to the integer-pipe result."""
    torch, pc2, ctx, N = env
    count = 2 * 148 * 128 + 37
    xs = W.uniform_below(N, count, 7)
    dx = pc2.ints_to_tiled(ctx, xs, 64)
    a = pc2.mont_sqr(ctx, N, dx, count, 9, pc2.ENGINE_IMAD)
    b = pc2.mont_sqr(ctx, N, dx, count, 9, pc2.ENGINE_TC)
    torch.cuda.synchronize()
    assert torch.equal(pc2.unpack(ctx, a, count, 64), pc2.unpack(ctx, b, count, 64))
    idx = [0, 127, 128, count // 2, count - 1]
    got = pc2.tiled_to_ints(ctx, b, count, 64)
    assert [got[i] for i in idx] == _expect(N, [xs[i] for i in idx], 9)
    assert ctx.status() == 0
