"""GPU parity of the Paillier kernels against the CPU oracle (bit-exact).

Inputs are seeded (paper_2601_14980_b300.workloads); both sides draw r from
the same published Philox4x32-10 definition, implemented independently.
Sizes span several 32-element tiles with a ragged tail; the full-size
2048-bit workload (2^20 plaintexts) is checked on sampled elements."""
import numpy as np
import pytest

from oracle import paillier as O
from paper_2601_14980_b300 import workloads as W

pytestmark = pytest.mark.gpu

SEED, STREAM = 0x5EED5EED, 7


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2601_14980_b300 import pc2

    ctx = pc2.Context(0)
    return torch, pc2, ctx


def _keys(pc2, nbits, seed=1):
    p, q = W.primes(nbits, seed)
    return pc2.Key.from_primes(p, q), O.derive_key(p, q)


def _oracle_ct(ko, m, e0=0, seed=SEED, stream=STREAM):
    return O.encrypt(ko, [int(x) for x in m], [O.r_of(ko, seed, stream, e0 + e) for e in range(len(m))])


@pytest.mark.parametrize("nbits,count", [(256, 77), (512, 70), (1024, 40)])
def test_encrypt_crt_and_public_bit_exact(env, nbits, count):
    torch, pc2, ctx = env
    kg, ko = _keys(pc2, nbits)
    m = W.plaintexts_u64(count, seed=nbits)
    m[0], m[1] = 0, np.uint64(2**64 - 1)
    dm = torch.from_numpy(m.view(np.int64)).cuda()
    ref = _oracle_ct(ko, m, e0=5)
    ct = pc2.encrypt(ctx, kg, dm, SEED, STREAM, e0=5)
    assert pc2.tiled_to_ints(ctx, ct, count, 2 * kg.limbs) == ref
    ctp = pc2.encrypt(ctx, kg, dm, SEED, STREAM, e0=5, public=True)
    assert pc2.tiled_to_ints(ctx, ctp, count, 2 * kg.limbs) == ref
    kpub = kg.public()
    ctq = pc2.encrypt(ctx, kpub, dm, SEED, STREAM, e0=5)
    assert pc2.tiled_to_ints(ctx, ctq, count, 2 * kg.limbs) == ref
    assert ctx.status() == 0


@pytest.mark.parametrize("nbits,count", [(256, 65), (512, 33), (1024, 40)])
def test_decrypt_bit_exact(env, nbits, count):
    torch, pc2, ctx = env
    kg, ko = _keys(pc2, nbits, seed=2)
    # full-width plaintexts in [0, n), encrypted by the oracle
    m = W.uniform_below(ko.n, count, 3) + [0, 1, ko.n - 1]
    cnt = len(m)
    c = O.encrypt(ko, m, [O.r_of(ko, 9, 1, e) for e in range(cnt)])
    dct = pc2.ints_to_tiled(ctx, c, 2 * kg.limbs)
    dm = pc2.decrypt(ctx, kg, dct, cnt)
    assert pc2.tiled_to_ints(ctx, dm, cnt, kg.limbs) == m
    with pytest.raises(pc2.Pc2Error):
        pc2.decrypt(ctx, kg.public(), dct, cnt)


def test_encrypt_wide_and_range_flag(env):
    torch, pc2, ctx = env
    kg, ko = _keys(pc2, 512, seed=3)
    m = W.uniform_below(ko.n, 45, 4) + [ko.n - 1]
    dmw = pc2.ints_to_tiled(ctx, m, kg.limbs)
    ct = pc2.encrypt_wide(ctx, kg, dmw, len(m), SEED, STREAM)
    assert pc2.tiled_to_ints(ctx, ct, len(m), 2 * kg.limbs) == _oracle_ct(ko, m)
    assert ctx.status() == 0
    bad = pc2.ints_to_tiled(ctx, [ko.n], kg.limbs)
    pc2.encrypt_wide(ctx, kg, bad, 1, SEED, STREAM)
    assert ctx.status() & pc2.ST_RANGE


@pytest.mark.parametrize("nbits", [256, 1024])
def test_hom_add_sum_scal(env, nbits):
    torch, pc2, ctx = env
    kg, ko = _keys(pc2, nbits, seed=4)
    cnt = 37
    groups = [O.encrypt(ko, W.uniform_below(ko.n, cnt, 10 + g), [O.r_of(ko, 3, g, e) for e in range(cnt)])
              for g in range(35)]
    L2 = 2 * kg.limbs
    dg = [pc2.ints_to_tiled(ctx, grp, L2) for grp in groups]
    out = pc2.hom_add(ctx, kg, dg[0], dg[1], cnt)
    assert pc2.tiled_to_ints(ctx, out, cnt, L2) == O.hom_add(ko, groups[0], groups[1])
    for G in (1, 3, 35):   # 35 > 32 operands: chained launches
        stacked = torch.cat(dg[:G])
        out = pc2.hom_sum(ctx, kg, stacked, G, cnt)
        assert pc2.tiled_to_ints(ctx, out, cnt, L2) == O.hom_sum(ko, groups[:G]), G
    k = np.array([0, 1, 2, 3, 2**64 - 1] + W.uniform_below(2**40, cnt - 5, 5), dtype=np.uint64)
    dk = torch.from_numpy(k.view(np.int64)).cuda()
    out = pc2.hom_scal(ctx, kg, dg[0], dk, cnt)
    assert pc2.tiled_to_ints(ctx, out, cnt, L2) == O.hom_scal(ko, groups[0], [int(x) for x in k])


def test_empty_and_single(env):
    torch, pc2, ctx = env
    kg, ko = _keys(pc2, 256, seed=5)
    dm = torch.zeros(1, dtype=torch.int64, device="cuda")
    out = pc2.empty_tiled(1, 2 * kg.limbs)
    assert pc2._encrypt(ctx.h, kg.h, dm.data_ptr(), 0, 1, 1, 0, out.data_ptr(), None) == 0
    ct = pc2.encrypt(ctx, kg, dm, SEED, STREAM)
    assert pc2.tiled_to_ints(ctx, ct, 1, 2 * kg.limbs) == _oracle_ct(ko, [0])


def test_full_size_2048_sampled(env):
    """2^20 plaintexts at 2048-bit n (the benchmark's launch configuration):
    encrypt, aggregate 16 groups of 2^16, decrypt; check sampled elements."""
    torch, pc2, ctx = env
    kg = pc2.Key.generate(2048, 2026)
    e = kg.export()
    ko = O.derive_key(e["p"], e["q"])
    N, G = 1 << 20, 16
    m = W.plaintexts_u64(N, seed=7)
    dm = torch.from_numpy(m.view(np.int64)).cuda()
    L2 = 2 * kg.limbs
    ct = torch.empty(G * pc2.tiled_words(N // G, L2), dtype=torch.int32, device="cuda")
    for g in range(G):   # group g = elements [g N/G, (g+1) N/G), r counters continue across groups
        seg = ct[g * pc2.tiled_words(N // G, L2):(g + 1) * pc2.tiled_words(N // G, L2)]
        pc2.encrypt(ctx, kg, dm[g * (N // G):(g + 1) * (N // G)], SEED, STREAM, e0=g * (N // G), out=seg)
    agg = pc2.hom_sum(ctx, kg, ct, G, N // G)
    dec = pc2.decrypt(ctx, kg, agg, N // G)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    idx = sorted(set([0, N // G - 1] + rng.integers(0, N // G, 6).tolist()))
    canon = pc2.unpack(ctx, ct[: pc2.tiled_words(N // G, L2)], N // G, L2).cpu().numpy().view(np.uint32)
    for i in idx[:3]:
        ref = _oracle_ct(ko, [m[i]], e0=i)[0]
        assert int.from_bytes(canon[i * L2:(i + 1) * L2].tobytes(), "little") == ref
    decw = pc2.unpack(ctx, dec, N // G, kg.limbs).cpu().numpy().view(np.uint32)
    for i in idx:
        expect = sum(int(m[g * (N // G) + i]) for g in range(G)) % ko.n
        assert int.from_bytes(decw[i * kg.limbs:(i + 1) * kg.limbs].tobytes(), "little") == expect


@pytest.mark.parametrize("nbits", [256, 512, 1024, 2048])
def test_lanes_and_windows_bit_identical(env, nbits):
    """Every built lanes-per-element count and window width computes the same ciphertexts and plaintexts."""
    torch, pc2, ctx = env
    kg, ko = _keys(pc2, nbits, seed=6)
    count = 45
    m = W.plaintexts_u64(count, seed=nbits + 1)
    dm = torch.from_numpy(m.view(np.int64)).cuda()
    ref = _oracle_ct(ko, m)            # every element, lanes of both tiles
    L2 = 2 * kg.limbs
    try:
        for lanes, w, split in [(l, w, s) for l in (1, 2, 4, 8) for w in (0, 4, 6) for s in (1, 2)]:
            pc2.set_lanes(ctx, lanes)
            pc2.set_split(ctx, split)      # 1: halves one after the other, 2: in parallel
            ctx.set_window(w)
            try:
                ct = pc2.encrypt(ctx, kg, dm, SEED, STREAM)
            except pc2.Pc2Error as e:
                assert e.code == -8 and (lanes == 8 and kg.limbs == 8)  # not built for this size
                continue
            got = pc2.tiled_to_ints(ctx, ct, count, L2)
            assert got == ref, (lanes, w, split)
            dec = pc2.tiled_to_ints(ctx, pc2.decrypt(ctx, kg, ct, count), count, kg.limbs)
            assert dec == [int(x) for x in m], (lanes, w, split)
    finally:
        pc2.set_lanes(ctx, 0)
        pc2.set_split(ctx, 0)
        ctx.set_window(0)


def test_autotune_records_and_stays_exact(env):
    torch, pc2, ctx = env
    kg, ko = _keys(pc2, 1024, seed=7)
    res = pc2.autotune(ctx, kg, 300)
    assert res["encrypt"][0] in (1, 2, 4, 8) and 4 <= res["encrypt"][1] <= 6 and res["encrypt"][2] in (0, 1)
    assert res["decrypt"][0] in (1, 2, 4, 8) and 4 <= res["decrypt"][1] <= 6 and res["decrypt"][2] in (0, 1)
    m = W.plaintexts_u64(300, seed=8)
    ct = pc2.encrypt(ctx, kg, torch.from_numpy(m.view(np.int64)).cuda(), SEED, STREAM)
    assert pc2.tiled_to_ints(ctx, ct, 3, 2 * kg.limbs) == _oracle_ct(ko, m[:3])


def test_4096_bit_paths_bit_exact(env):
    """4096-bit n, the largest key of the paper's evaluation: key-owner
    encryption at every built lane count with the CRT halves one after the
    other and in parallel, the public path, decryption (64-bit and full-width
    plaintexts) and the homomorphic operations, against the oracle."""
    torch, pc2, ctx = env
    kg, ko = _keys(pc2, 4096, seed=4)
    assert kg.limbs == 128
    count = 34                      # one full tile and a ragged tail
    m = W.plaintexts_u64(count, seed=41)
    m[0], m[1] = 0, np.uint64(2**64 - 1)
    dm = torch.from_numpy(m.view(np.int64)).cuda()
    ref = _oracle_ct(ko, m, e0=3)
    L2 = 2 * kg.limbs
    try:
        for lanes in (2, 4, 8):
            for split in (1, 2):
                pc2.set_lanes(ctx, lanes)
                pc2.set_split(ctx, split)
                ct = pc2.encrypt(ctx, kg, dm, SEED, STREAM, e0=3)
                assert pc2.tiled_to_ints(ctx, ct, count, L2) == ref, (lanes, split)
                dec = pc2.tiled_to_ints(ctx, pc2.decrypt(ctx, kg, ct, count), count, kg.limbs)
                assert dec == [int(x) for x in m], (lanes, split)
    finally:
        pc2.set_lanes(ctx, 0)
        pc2.set_split(ctx, 0)
    ctp = pc2.encrypt(ctx, kg, dm[:5], SEED, STREAM, e0=3, public=True)
    assert pc2.tiled_to_ints(ctx, ctp, 5, L2) == ref[:5]
    mw = W.uniform_below(ko.n, 3, 5) + [ko.n - 1]
    cw = O.encrypt(ko, mw, [O.r_of(ko, 9, 1, e) for e in range(len(mw))])
    dcw = pc2.ints_to_tiled(ctx, cw, L2)
    assert pc2.tiled_to_ints(ctx, pc2.decrypt(ctx, kg, dcw, len(mw)), len(mw), kg.limbs) == mw
    a, b = pc2.ints_to_tiled(ctx, ref[:4], L2), dcw
    assert pc2.tiled_to_ints(ctx, pc2.hom_add(ctx, kg, a, b, 4), 4, L2) == O.hom_add(ko, ref[:4], cw)
    k = np.array([0, 1, 3, 2**64 - 1], dtype=np.uint64)
    out = pc2.hom_scal(ctx, kg, a, torch.from_numpy(k.view(np.int64)).cuda(), 4)
    assert pc2.tiled_to_ints(ctx, out, 4, L2) == O.hom_scal(ko, ref[:4], [int(x) for x in k])
    assert ctx.status() == 0


@pytest.mark.parametrize("nbits,count", [(512, 37), (2048, 9), (4096, 3)])
def test_hom_scal_wide_bit_exact(env, nbits, count):
    """Definition 2 with full-width scalars (the plain power mod n^2) against the oracle."""
    torch, pc2, ctx = env
    kg, ko = _keys(pc2, nbits, seed=8)
    L2 = 2 * kg.limbs
    c = O.encrypt(ko, W.uniform_below(ko.n, count, 12), [O.r_of(ko, 4, 4, e) for e in range(count)])
    ks = [0, 1, 2**nbits - 1] + W.uniform_below(ko.n, count - 3, 13)
    dc, dk = pc2.ints_to_tiled(ctx, c, L2), pc2.ints_to_tiled(ctx, ks, kg.limbs)
    out = pc2.hom_scal_wide(ctx, kg, dc, dk, count)
    assert pc2.tiled_to_ints(ctx, out, count, L2) == O.hom_scal_wide(ko, c, ks)
    for w in (4, 6):
        ctx.set_window(w)
        try:
            out = pc2.hom_scal_wide(ctx, kg, dc, dk, count)
        finally:
            ctx.set_window(0)
        assert pc2.tiled_to_ints(ctx, out, 2, L2) == O.hom_scal_wide(ko, c[:2], ks[:2]), w


@pytest.mark.parametrize("nbits", [256, 512, 1024, 2048])
def test_n2_ops_lanes_bit_identical(env, nbits):
    """Public encryption, products, 64-bit and full-width scalar powers mod n^2
    give the oracle's results at every lane count (forced; sizes without a
    lane count fall back to the automatic choice)."""
    torch, pc2, ctx = env
    kg, ko = _keys(pc2, nbits, seed=9)
    count, L2 = 37, 2 * kg.limbs
    m = W.plaintexts_u64(count, seed=nbits + 3)
    dm = torch.from_numpy(m.view(np.int64)).cuda()
    ref_ct = _oracle_ct(ko, m)
    c2 = O.encrypt(ko, W.uniform_below(ko.n, count, 14), [O.r_of(ko, 2, 2, e) for e in range(count)])
    k64 = np.array([0, 1, 2**64 - 1] + W.uniform_below(2**64, count - 3, 15), dtype=np.uint64)
    kw = [0, 1, 2**nbits - 1] + W.uniform_below(ko.n, count - 3, 16)
    ref_add = O.hom_add(ko, ref_ct, c2)
    ref_sum = O.hom_sum(ko, [ref_ct, c2, ref_ct])
    ref_scal = O.hom_scal(ko, ref_ct, [int(x) for x in k64])
    ref_wide = O.hom_scal_wide(ko, ref_ct, kw)
    d1, d2 = pc2.ints_to_tiled(ctx, ref_ct, L2), pc2.ints_to_tiled(ctx, c2, L2)
    dk64 = torch.from_numpy(k64.view(np.int64)).cuda()
    dkw = pc2.ints_to_tiled(ctx, kw, kg.limbs)
    try:
        for lanes in (1, 2, 4, 8):
            pc2.set_lanes(ctx, lanes)
            ct = pc2.encrypt(ctx, kg, dm, SEED, STREAM, public=True)
            assert pc2.tiled_to_ints(ctx, ct, count, L2) == ref_ct, lanes
            assert pc2.tiled_to_ints(ctx, pc2.hom_add(ctx, kg, d1, d2, count), count, L2) == ref_add, lanes
            out = pc2.hom_sum(ctx, kg, torch.cat([d1, d2, d1]), 3, count)
            assert pc2.tiled_to_ints(ctx, out, count, L2) == ref_sum, lanes
            out = pc2.hom_scal(ctx, kg, d1, dk64, count)
            assert pc2.tiled_to_ints(ctx, out, count, L2) == ref_scal, lanes
            out = pc2.hom_scal_wide(ctx, kg, d1, dkw, count)
            assert pc2.tiled_to_ints(ctx, out, count, L2) == ref_wide, lanes
    finally:
        pc2.set_lanes(ctx, 0)
    assert ctx.status() == 0
