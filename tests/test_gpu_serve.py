"""GPU tests of the serving form (include/pc2.h, pc2_server_*): every
request's result equals the per-operation entry point's (pc2_encrypt,
pc2_decrypt, pc2_hom_sum) -- alone, in a mix of concurrent requests, under a
tight memory arena, and on the plain per-request path -- and sampled results
equal the oracle's."""
import numpy as np
import pytest

from oracle import paillier as O
from paper_2601_14980_b300 import workloads as W

pytestmark = pytest.mark.gpu

SEED = 99


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2601_14980_b300 import pc2

    return torch, pc2, pc2.Context(0)


def _keys(pc2, nbits, seed=2):
    p, q = W.primes(nbits, seed)
    return pc2.Key.from_primes(p, q), O.derive_key(p, q)


class _Req:
    """One request: its host buffers and the expected output (device entry points)."""

    def __init__(self, env, kg, op, count, rng, groups=1, stream=0, e0=0):
        torch, pc2, ctx = env
        L = kg.limbs
        self.op, self.count, self.groups, self.stream, self.e0 = op, count, groups, stream, e0
        m = W.plaintexts_u64(count, seed=int(rng.integers(1 << 30)))
        dm = torch.from_numpy(m.view(np.int64)).cuda()
        if op == pc2.OP_ENCRYPT:
            self.h_in = torch.from_numpy(m.view(np.int64)).pin_memory()
            want = pc2.encrypt(ctx, kg, dm, SEED, stream, e0)
            self.out_words = pc2.tiled_words(count, 2 * L)
        elif op == pc2.OP_DECRYPT:
            ct = pc2.encrypt(ctx, kg, dm, SEED + 1, stream, e0)
            self.h_in = ct.cpu().pin_memory()
            want = pc2.decrypt(ctx, kg, ct, count)
            self.out_words = pc2.tiled_words(count, L)
        else:
            cts = [pc2.encrypt(ctx, kg, dm, SEED + 2 + g, stream, e0) for g in range(groups)]
            allc = torch.cat([c[:pc2.tiled_words(count, 2 * L)] for c in cts])
            self.h_in = allc.cpu().pin_memory()
            want = pc2.hom_sum(ctx, kg, allc, groups, count)
            self.out_words = pc2.tiled_words(count, 2 * L)
        self.out_limbs = L if op == pc2.OP_DECRYPT else 2 * L
        self.pc2, self.ctx = pc2, ctx
        # compare element words only (a tile's padding slots are never written)
        self.want = pc2.unpack(ctx, want, count, self.out_limbs).cpu()
        torch.cuda.synchronize()
        self.h_out = torch.zeros(self.out_words, dtype=torch.int32).pin_memory()

    def submit(self, srv):
        self.h_out.zero_()
        self.t = srv.submit(self.op, self.h_in, self.count, self.h_out, groups=self.groups, seed=SEED,
                            stream=self.stream, e0=self.e0)
        return self.t

    def ok(self):
        import torch

        got = self.pc2.unpack(self.ctx, self.h_out.cuda(), self.count, self.out_limbs).cpu()
        return torch.equal(got, self.want)


def _mix(env, kg, n, rng, lo=1, hi=3000):
    torch, pc2, ctx = env
    out = []
    for i in range(n):
        op = [pc2.OP_ENCRYPT, pc2.OP_DECRYPT, pc2.OP_AGGREGATE][i % 3]
        count = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        out.append(_Req(env, kg, op, count, rng, groups=int(rng.integers(2, 7)), stream=i + 1, e0=int(rng.integers(0, 1000))))
    return out


def test_each_result_is_the_same_alone_and_in_the_mix(env):
    torch, pc2, ctx = env
    kg, ko = _keys(pc2, 512)
    rng = np.random.default_rng(0)
    reqs = _mix(env, kg, 18, rng)
    probe = _Req(env, kg, pc2.OP_ENCRYPT, 700, rng, stream=77, e0=5)
    srv = pc2.Server(ctx, kg, arena_bytes=256 << 20)
    probe.submit(srv)
    srv.wait(probe.t)
    alone = probe.h_out.clone()
    assert probe.ok()
    # the same request again, submitted in the middle of a burst of others
    ts = [r.submit(srv) for r in reqs[:9]] + [probe.submit(srv)] + [r.submit(srv) for r in reqs[9:]]
    for t in ts:
        srv.wait(t)
    assert torch.equal(probe.h_out, alone)
    for r in reqs:
        assert r.ok(), (r.op, r.count)
    st = srv.stats()
    assert st["completed"] == 20 and st["steps"] >= 2
    srv.close()
    assert ctx.status() == 0
    # sampled against the oracle: the probe's ciphertexts
    got = pc2.tiled_to_ints(ctx, alone.cuda(), 700, 2 * kg.limbs)
    m = probe.h_in.numpy().view(np.uint64)
    for i in (0, 350, 699):
        assert got[i] == O.encrypt(ko, [int(m[i])], [O.r_of(ko, SEED, 77, 5 + i)])[0]


def test_admission_by_memory_and_plain_path(env):
    torch, pc2, ctx = env
    kg, _ = _keys(pc2, 512)
    rng = np.random.default_rng(1)
    reqs = _mix(env, kg, 12, rng, lo=200, hi=4000)
    need = max(r.h_in.numel() * r.h_in.element_size() + r.out_words * 4 for r in reqs)
    arena = need + (1 << 16)               # room for about one request at a time
    for mode in (0, 1):
        srv = pc2.Server(ctx, kg, arena_bytes=arena, mode=mode)
        ts = [r.submit(srv) for r in reqs]
        lats = [srv.wait(t) for t in ts]
        assert all(r.ok() for r in reqs), mode
        assert all(x > 0 for x in lats)
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["arena_peak"] <= arena
        srv.close()
    assert ctx.status() == 0


def test_small_and_large_lanes_and_2048_bit(env):
    torch, pc2, ctx = env
    kg, ko = _keys(pc2, 2048)
    rng = np.random.default_rng(2)
    reqs = [_Req(env, kg, pc2.OP_ENCRYPT, 70, rng, stream=3),          # 8 lanes per element
            _Req(env, kg, pc2.OP_ENCRYPT, 300, rng, stream=4, e0=9),   # one lane per element (small_request below)
            _Req(env, kg, pc2.OP_DECRYPT, 260, rng, stream=5),
            _Req(env, kg, pc2.OP_AGGREGATE, 100, rng, groups=16, stream=6)]
    srv = pc2.Server(ctx, kg, arena_bytes=64 << 20, small_request=128)
    ts = [r.submit(srv) for r in reqs]
    for t in ts:
        srv.wait(t)
    assert all(r.ok() for r in reqs)
    srv.close()
    got = pc2.tiled_to_ints(ctx, reqs[0].h_out.cuda(), 70, 2 * kg.limbs)
    m = reqs[0].h_in.numpy().view(np.uint64)
    assert got[69] == O.encrypt(ko, [int(m[69])], [O.r_of(ko, SEED, 3, 69)])[0]
    assert ctx.status() == 0


def test_rejects_what_cannot_fit(env):
    torch, pc2, ctx = env
    kg, _ = _keys(pc2, 512)
    srv = pc2.Server(ctx, kg, arena_bytes=1 << 16)
    h_in = torch.zeros(10000, dtype=torch.int64)
    h_out = torch.zeros(pc2.tiled_words(10000, 2 * kg.limbs), dtype=torch.int32)
    with pytest.raises(pc2.Pc2Error):
        srv.submit(pc2.OP_ENCRYPT, h_in, 10000, h_out)
    with pytest.raises(pc2.Pc2Error):
        srv.submit(pc2.OP_AGGREGATE, h_in, 10, h_out, groups=1)
    srv.close()


def test_aggregate_from_a_strided_pool(env):
    torch, pc2, ctx = env
    kg, _ = _keys(pc2, 512)
    L2 = 2 * kg.limbs
    m = W.plaintexts_u64(500, seed=5)
    dm = torch.from_numpy(m.view(np.int64)).cuda()
    pool = torch.cat([pc2.encrypt(ctx, kg, dm, SEED + g, g, 0)[:pc2.tiled_words(500, L2)] for g in range(3)])
    stride = pc2.tiled_words(500, L2)
    count = 100
    packed = torch.cat([pool[g * stride:g * stride + pc2.tiled_words(count, L2)] for g in range(3)])
    want = pc2.unpack(ctx, pc2.hom_sum(ctx, kg, packed, 3, count), count, L2).cpu()
    h_in = pool.cpu().pin_memory()
    h_out = torch.zeros(pc2.tiled_words(count, L2), dtype=torch.int32).pin_memory()
    srv = pc2.Server(ctx, kg, arena_bytes=16 << 20)
    srv.wait(srv.submit(pc2.OP_AGGREGATE, h_in, count, h_out, groups=3, h_stride=stride))
    srv.close()
    assert torch.equal(pc2.unpack(ctx, h_out.cuda(), count, L2).cpu(), want)


def test_concurrent_submitters(env):
    """Four host threads submit and wait at the same time; every result equals the entry point's."""
    import threading

    torch, pc2, ctx = env
    kg, _ = _keys(pc2, 512)
    rng = np.random.default_rng(3)
    reqs = _mix(env, kg, 16, rng, lo=20, hi=1500)
    srv = pc2.Server(ctx, kg, arena_bytes=64 << 20)
    errors = []

    def worker(chunk):
        try:
            ts = [r.submit(srv) for r in chunk]
            for t in ts:
                srv.wait(t)
        except Exception as e:  # noqa: BLE001 - reported by the main thread
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(reqs[i::4],)) for i in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join(timeout=300)
    assert not errors
    assert all(r.ok() for r in reqs)
    assert srv.stats()["completed"] == len(reqs)
    srv.close()
