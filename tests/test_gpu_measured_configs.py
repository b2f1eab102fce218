"""GPU parity on the configurations the benchmark times, against the oracle.

* The memory-bound steps (quantize Gamma1/Gamma2 of Eq. (et21) with and
  without negation, the inverse quantization, the z/v update of Eqs. (ty32),
  (u78)) on 2^21 + 37 elements: large enough that every thread of the
  launch runs the four-loads-in-flight loop and then the ragged tail loop.
* The benchmark's Paillier step exactly as bench.py launches it: one
  pc2_encrypt of 2^20 quantized plaintexts at 2048-bit n (key-owner CRT
  path, default lane choice), the 16-group product and the CRT decryption of
  the 2^16 aggregates.  256 ciphertexts, spread over all 32 lanes of a warp at
  eight positions from the first persistent pass to the last tile, are
  compared with oracle.encrypt (Eq. (itq1)); every aggregate's decryption is
  compared with the exact group sum.
* Key-owner encryption of full-width plaintexts (Eq. (itq1), m in Z_n) at
  1024, 2048 and 4096 bits and decryption of full-width plaintexts
  (Sec. III-C) at 2048 bits.

The oracle runs in a thread pool: its C calls release the interpreter lock."""
import concurrent.futures as cf
import os

import numpy as np
import pytest

from oracle import admm as OA
from oracle import paillier as O
from paper_2601_14980_b300 import workloads as W

pytestmark = pytest.mark.gpu

QP = OA.QParams(zmin=-8.0, zmax=8.0, log2_scale=24)
N_BW = (1 << 21) + 37


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2601_14980_b300 import pc2

    return torch, pc2, pc2.Context(0)


def _pool_encrypt(ko, m, e0s, seed, stream):
    """oracle.encrypt of m[i] with r drawn for counter e0s[i], in parallel chunks."""
    m, e0s = [int(x) for x in m], [int(e) for e in e0s]
    workers = max(1, min(32, os.cpu_count() or 1))
    chunks = [list(range(i, len(m), workers)) for i in range(workers)]

    def job(ix):
        return ix, O.encrypt(ko, [m[i] for i in ix], [O.r_of(ko, seed, stream, e0s[i]) for i in ix])

    out = [None] * len(m)
    with cf.ThreadPoolExecutor(workers) as ex:
        for ix, cts in ex.map(job, [c for c in chunks if c]):
            for i, c in zip(ix, cts):
                out[i] = c
    return out


# ------------------------------------------------------------------ memory-bound steps


def _bw_input(seed):
    rng = np.random.default_rng(seed)
    u = rng.standard_normal(N_BW)
    u[:6] = [QP.zmin, QP.zmax, 0.0, -0.0, QP.zmin + 2.0 ** -25, QP.zmax - 2.0 ** -25]
    # exact half-way points of both quantizers, spread over the vector
    j = rng.integers(0, 1 << 20, 4096)
    pos = rng.integers(6, N_BW, 4096)
    u[pos[:2048]] = QP.zmin + (2 * j[:2048] + 1) * 2.0 ** -25
    u[pos[2048:]] = QP.zmin + (2 * j[2048:] + 1) * 2.0 ** -49
    return u


@pytest.mark.parametrize("gamma", [2, 1])
@pytest.mark.parametrize("negate", [False, True])
def test_quantize_and_dequantize_full_loop(env, gamma, negate):
    """Eq. (et21) element by element against the oracle; the inverse
    quantization against q / S^k + zmin, the exact rational rounded once."""
    torch, pc2, ctx = env
    u = _bw_input(11 + gamma)
    du = torch.from_numpy(u).cuda()
    q = pc2.quantize(ctx, du, QP.zmin, QP.zmax, QP.log2_scale, gamma, negate=negate)
    src = -u if negate else u
    want = (OA.gamma2 if gamma == 2 else OA.gamma1)(src, QP)
    got = q.cpu().numpy()
    assert np.array_equal(got, want)
    assert ctx.status() == 0
    back = pc2.dequantize(ctx, q, QP.zmin, QP.log2_scale, gamma).cpu().numpy()
    k = QP.log2_scale * (2 if gamma == 1 else 1)
    # q < 2^53, so q 2^-k is exact in float64 and the one addition rounds the
    # exact rational q / 2^k + zmin
    ref = want.astype(np.float64) * 2.0 ** -k + QP.zmin
    assert np.array_equal(back, ref)
    from fractions import Fraction

    for i in list(range(8)) + [N_BW // 2, N_BW - 1]:
        assert back[i] == float(Fraction(int(want[i]), 2 ** k) + Fraction(QP.zmin))


def test_zv_update_full_loop(env):
    """Eqs. (ty32), (u78) on 2^21 + 37 elements, bit-exact, with exact +-kappa
    edges and dead-zone values sprinkled through the vector."""
    torch, pc2, ctx = env
    rng = np.random.default_rng(21)
    kappa = 0.01
    x = rng.standard_normal(N_BW) * 0.02
    v = rng.standard_normal(N_BW) * 0.02
    pos = rng.integers(0, N_BW, 3000)
    x[pos[:1000]], v[pos[:1000]] = kappa, 0.0
    x[pos[1000:2000]], v[pos[1000:2000]] = -kappa, 0.0
    x[pos[2000:]] = 0.0
    z_ref = OA.soft_threshold(v + x, kappa)
    v_ref = v + x - z_ref
    dx, dz, dv = (torch.from_numpy(a.copy()).cuda() for a in (x, np.full(N_BW, 7.0), v))
    pc2.zv_update(ctx, dx, dz, dv, kappa)
    assert np.array_equal(dz.cpu().numpy(), z_ref)
    assert np.array_equal(dv.cpu().numpy(), v_ref)


# ------------------------------------------------------------------ the benchmark's Paillier step


def test_bench_step_2048_bits_spread_samples(env):
    torch, pc2, ctx = env
    N, G, SEED, STREAM = 1 << 20, 16, 0xB300, 1      # the benchmark's workload and r stream
    key = pc2.Key.generate(2048, 2026)
    e = key.export()
    ko = O.derive_key(e["p"], e["q"])
    m = W.plaintexts_u64(N, seed=7)
    dm = torch.from_numpy(m.view(np.int64)).cuda()
    L2 = 2 * key.limbs
    per = N // G
    ct = torch.empty(pc2.tiled_words(N, L2), dtype=torch.int32, device="cuda")
    agg = torch.empty(pc2.tiled_words(per, L2), dtype=torch.int32, device="cuda")
    dec = torch.empty(pc2.tiled_words(per, key.limbs), dtype=torch.int32, device="cuda")
    pc2.encrypt(ctx, key, dm, SEED, STREAM, e0=0, out=ct)
    pc2.hom_sum(ctx, key, ct, G, per, out=agg)
    pc2.decrypt(ctx, key, agg, per, out=dec)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    # 32 lanes at eight tile-aligned positions: first pass, later persistent
    # passes (a pass covers a few times 10^4 elements), the last tile
    anchors = [0, 4096, 60000, 300000, 600000, 900000, 1029984, N - 32]
    idx = sorted({a + lane for a in anchors for lane in range(32)})
    assert len(idx) == 256
    canon = pc2.unpack(ctx, ct, N, L2).cpu().numpy().view(np.uint32).reshape(N, L2)
    got = [int.from_bytes(canon[i].tobytes(), "little") for i in idx]
    want = _pool_encrypt(ko, [m[i] for i in idx], idx, SEED, STREAM)
    bad = [i for i, g, w in zip(idx, got, want) if g != w]
    assert not bad, "ciphertexts differ from the oracle at %s" % bad[:8]
    # every aggregate: sum of its 16 group members (< n, so no reduction)
    w = pc2.unpack(ctx, dec, per, key.limbs).cpu().numpy().view(np.uint32).reshape(per, key.limbs)
    assert not w[:, 3:].any()
    got_sum = [int(a) | (int(b) << 32) | (int(c) << 64) for a, b, c in zip(w[:, 0], w[:, 1], w[:, 2])]
    ms = m.reshape(G, per)
    want_sum = [sum(int(ms[g, i]) for g in range(G)) for i in range(per)]
    assert got_sum == want_sum


# ------------------------------------------------------------------ full-width plaintexts


@pytest.mark.parametrize("nbits,count", [(1024, 40), (2048, 36), (4096, 34)])
def test_encrypt_wide_against_oracle(env, nbits, count):
    """Key-owner encryption of plaintexts in [0, n): one full tile and a ragged tail."""
    torch, pc2, ctx = env
    p, q = W.primes(nbits, 12)
    kg, ko = pc2.Key.from_primes(p, q), O.derive_key(p, q)
    m = [0, 1, ko.n - 1] + W.uniform_below(ko.n, count - 3, nbits + 5)
    dmw = pc2.ints_to_tiled(ctx, m, kg.limbs)
    ct = pc2.encrypt_wide(ctx, kg, dmw, count, 99, 4, e0=11)
    got = pc2.tiled_to_ints(ctx, ct, count, 2 * kg.limbs)
    assert got == _pool_encrypt(ko, m, [11 + i for i in range(count)], 99, 4)
    assert ctx.status() == 0


def test_decrypt_full_width_2048(env):
    """Sec. III-C at 2048-bit n on plaintexts spanning [0, n), encrypted by the oracle."""
    torch, pc2, ctx = env
    p, q = W.primes(2048, 13)
    kg, ko = pc2.Key.from_primes(p, q), O.derive_key(p, q)
    m = [0, 1, 2, ko.n - 1, ko.n - 2] + W.uniform_below(ko.n, 36, 77)
    c = _pool_encrypt(ko, m, list(range(len(m))), 5, 6)
    dct = pc2.ints_to_tiled(ctx, c, 2 * kg.limbs)
    dm = pc2.decrypt(ctx, kg, dct, len(m))
    assert pc2.tiled_to_ints(ctx, dm, len(m), kg.limbs) == m
