"""GPU parity of the batched round (many edge nodes, mixed key sizes, one
persistent launch per round) against the oracle.

The design is orthonormal, so the oracle runs the quantized round over 1 x 1
blocks (oracle.admm.diag_setup; pinned against the general set-up and the
N_k x N_k block form in tests/test_oracle_admm.py).  Iterates are
bit-identical; ciphertexts are bit-identical given the same Philox draws
(r-stream (t << 8) | kind, counter = global element index, each node's own
key)."""
import numpy as np
import pytest

from oracle import admm as O
from oracle import paillier as P
from paper_2601_14980_b300 import workloads as W

pytestmark = pytest.mark.gpu

QP = O.QParams(zmin=-8.0, zmax=8.0, log2_scale=24)
SEED = 4242


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2601_14980_b300 import pc2

    return torch, pc2, pc2.Context(0)


def _keys(pc2, bits_list, seed=3):
    out = []
    for bits in bits_list:
        p, q = W.primes(bits, seed)
        out.append((pc2.Key.from_primes(p, q), P.derive_key(p, q)))
    return out


def _make(env, sizes, node_key, bits_list, lam=0.02, rho=1.0, seed=SEED, prob_seed=9):
    torch, pc2, ctx = env
    rng = np.random.default_rng(prob_seed)
    N = sum(sizes)
    x0 = np.where(rng.random(N) < 0.3, rng.standard_normal(N), 0.0)
    aty = x0 + 0.01 * rng.standard_normal(N)
    st = O.diag_setup(aty, rho)
    alpha = torch.from_numpy(np.array([a[0] for a in st.alpha])).cuda()
    bdiag = torch.from_numpy(np.array([b[0, 0] for b in st.Bbar])).cuda()
    keys = _keys(pc2, bits_list)
    bt = pc2.Batch(ctx, [k for k, _ in keys], sizes, node_key, alpha, bdiag, lam, rho, QP.zmin, QP.zmax,
                   QP.log2_scale, seed)
    return st, keys, bt


def _cts(env, bt, which, node, count):
    torch, pc2, ctx = env
    ptr, limbs = bt.ciphertexts(which, node)
    w = pc2.device_words(ptr, pc2.tiled_words(count, limbs))
    return pc2.tiled_to_ints(ctx, w, count, limbs)


# nodes of uneven sizes (several work items, ragged tiles, a single-element
# node) and all five key sizes, 3072 bits running four lanes per element
SIZES = [3, 140, 1, 37, 70, 9, 129, 2, 33]
NODE_KEY = [0, 1, 2, 3, 4, 0, 1, 3, 2]
BITS = [256, 512, 1024, 2048, 3072]


def test_batched_rounds_match_oracle_bit_exact(env):
    torch, pc2, ctx = env
    st, keys, bt = _make(env, SIZES, NODE_KEY, BITS)
    lam, rho, T = 0.02, 1.0, 3
    ref = O.quantized_admm(st, lam, rho, T, QP)
    offs = np.concatenate([[0], np.cumsum(SIZES)]).astype(int)
    b = O.gamma2(np.array([B[0, 0] for B in st.Bbar]), QP)
    c1 = O.gamma1(np.array([a[0] for a in st.alpha]), QP)
    for t in range(1, T + 1):
        bt.round(1)
        x, z, v, nxt = bt.get()
        assert nxt == t + 1
        assert np.array_equal(x.cpu().numpy(), ref.x[t - 1]), t
        assert np.array_equal(z.cpu().numpy(), ref.z[t - 1]), t
        assert np.array_equal(v.cpu().numpy(), ref.v[t - 1]), t
    assert ctx.status() == 0
    # ciphertexts of the last round on sampled elements of every node, with the node's own key
    zprev, vprev = ref.z[T - 2], ref.v[T - 2]
    zq, vq = O.gamma2(zprev, QP), O.gamma2(-vprev, QP)
    for k, n in enumerate(SIZES):
        kg, ko = keys[NODE_KEY[k]]
        ah, zh = _cts(env, bt, "alpha_hat", k, n), _cts(env, bt, "zhat", k, n)
        vh, xh = _cts(env, bt, "vhat", k, n), _cts(env, bt, "xhat", k, n)
        for i in sorted({0, n // 2, n - 1}):
            e = int(offs[k] + i)
            assert ah[i] == P.encrypt(ko, [int(c1[e])], [P.r_of(ko, SEED, O.stream_id(0, O.KIND_ALPHA), e)])[0]
            assert zh[i] == P.encrypt(ko, [int(zq[e])], [P.r_of(ko, SEED, O.stream_id(T, O.KIND_Z), e)])[0], (k, i)
            assert vh[i] == P.encrypt(ko, [int(vq[e])], [P.r_of(ko, SEED, O.stream_id(T, O.KIND_V), e)])[0], (k, i)
            s = P.hom_add(ko, [zh[i]], [vh[i]])
            assert xh[i] == P.hom_matvec(ko, [ah[i]], s, np.array([[b[e]]], dtype=np.uint64))[0], (k, i)
            assert P.decrypt(ko, [xh[i]])[0] == ref.D[T - 1][e]
    bt.close()


def test_per_node_path_is_bit_identical(env):
    torch, pc2, ctx = env
    _, _, b1 = _make(env, SIZES, NODE_KEY, BITS)
    _, _, b2 = _make(env, SIZES, NODE_KEY, BITS)
    b1.round(2)
    b2.round_per_node(1)
    b2.round(1)                      # the paths share the state and the round counter
    g1, g2 = b1.get(), b2.get()
    for u, w in zip(g1[:3], g2[:3]):
        assert torch.equal(u, w)
    assert g1[3] == g2[3] == 3
    for k, n in enumerate(SIZES):
        for which in ("zhat", "vhat", "xhat"):
            assert _cts(env, b1, which, k, n) == _cts(env, b2, which, k, n), (k, which)
    b1.reset()
    b1.round_per_node(2)
    g3 = b1.get()
    for u, w in zip(g1[:3], g3[:3]):
        assert torch.equal(u, w)
    b1.close()
    b2.close()


def test_autotuner_changes_no_state_and_no_result(env):
    torch, pc2, ctx = env
    st, keys, bt = _make(env, SIZES, NODE_KEY, BITS)
    ref = O.quantized_admm(st, 0.02, 1.0, 2, QP)
    bt.round(1)
    before = bt.get()
    res = bt.tune(sample_items=12)
    assert 1 <= res["ctas_per_sm"] <= 3 and set(res["window"]) == set(BITS)
    assert all(4 <= w <= 6 for w in res["window"].values())
    after = bt.get()
    for u, w in zip(before[:3], after[:3]):
        assert torch.equal(u, w)
    assert before[3] == after[3] == 2
    bt.round(1)
    x, z, v, _ = bt.get()
    assert np.array_equal(x.cpu().numpy(), ref.x[1]) and np.array_equal(z.cpu().numpy(), ref.z[1])
    assert ctx.status() == 0
    bt.close()


def test_one_key_size_and_single_node(env):
    torch, pc2, ctx = env
    st, keys, bt = _make(env, [300], [0], [1024])
    ref = O.quantized_admm(st, 0.02, 1.0, 2, QP)
    bt.round(2)
    x, z, v, _ = bt.get()
    assert np.array_equal(x.cpu().numpy(), ref.x[1]) and np.array_equal(v.cpu().numpy(), ref.v[1])
    assert bt.info()["items"] == 3
    bt.close()


def _check_round_cts(env, bt, keys, sizes, node_key, ref, T, nodes, picks):
    """Ciphertexts of round T on the picked elements of the given nodes against the oracle."""
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(int)
    zq, vq = O.gamma2(ref.z[T - 2], QP), O.gamma2(-ref.v[T - 2], QP)
    for k in nodes:
        n = sizes[k]
        kg, ko = keys[node_key[k]]
        zh, vh, xh = _cts(env, bt, "zhat", k, n), _cts(env, bt, "vhat", k, n), _cts(env, bt, "xhat", k, n)
        for i in picks(n):
            e = int(offs[k] + i)
            assert zh[i] == P.encrypt(ko, [int(zq[e])], [P.r_of(ko, SEED, O.stream_id(T, O.KIND_Z), e)])[0], (k, i)
            assert vh[i] == P.encrypt(ko, [int(vq[e])], [P.r_of(ko, SEED, O.stream_id(T, O.KIND_V), e)])[0], (k, i)
            assert P.decrypt(ko, [xh[i]])[0] == ref.D[T - 1][e], (k, i)


def test_forced_tensor_core_nodes_match_oracle(env):
    """With the engine forced to the tensor cores every 2048-bit node leaves the
    work list and runs node by node before the persistent launch of each round;
    iterates and ciphertexts stay those of the oracle."""
    torch, pc2, ctx = env
    pc2.set_engine(ctx, pc2.ENGINE_TC)
    try:
        st, keys, bt = _make(env, SIZES, NODE_KEY, BITS)
        G = {256: 128, 512: 128, 1024: 128, 2048: 128, 3072: 32}
        assert bt.info()["items"] == sum(-(-n // G[BITS[k]]) for n, k in zip(SIZES, NODE_KEY) if BITS[k] != 2048)
        T = 3
        ref = O.quantized_admm(st, 0.02, 1.0, T, QP)
        for t in range(1, T + 1):
            bt.round(1)
            x, z, v, nxt = bt.get()
            assert nxt == t + 1
            assert np.array_equal(x.cpu().numpy(), ref.x[t - 1]) and np.array_equal(v.cpu().numpy(), ref.v[t - 1])
        assert ctx.status() == 0
        nodes = [k for k in range(len(SIZES)) if BITS[NODE_KEY[k]] == 2048] + [0, 4]
        _check_round_cts(env, bt, keys, SIZES, NODE_KEY, ref, T, nodes, lambda n: sorted({0, n // 2, n - 1}))
        bt.close()
    finally:
        pc2.set_engine(ctx, -1)


def test_large_2048_node_on_tensor_cores_automatic(env):
    """A 2048-bit node of PC2_TC_MIN_COUNT + 16 elements (tensor-core engine, a
    ragged last tile) beside a small 1024-bit node (the persistent launch):
    iterates equal the oracle's and the per-node path's; sampled ciphertexts
    of both nodes equal the oracle's."""
    torch, pc2, ctx = env
    sizes, node_key = [16384 + 16, 50], [0, 1]
    st, keys, bt = _make(env, sizes, node_key, [2048, 1024])
    assert bt.info()["items"] == 1
    T = 2
    ref = O.quantized_admm(st, 0.02, 1.0, T, QP)
    bt.round(T)
    x, z, v, nxt = bt.get()
    assert nxt == T + 1 and ctx.status() == 0
    assert np.array_equal(x.cpu().numpy(), ref.x[T - 1]) and np.array_equal(z.cpu().numpy(), ref.z[T - 1])
    assert np.array_equal(v.cpu().numpy(), ref.v[T - 1])
    _check_round_cts(env, bt, keys, sizes, node_key, ref, T, [0, 1], lambda n: sorted(i for i in {0, 127, 128, n // 2, n - 1} if i < n))
    _, _, b2 = _make(env, sizes, node_key, [2048, 1024])
    b2.round_per_node(T)
    g = b2.get()
    assert torch.equal(g[0], x) and torch.equal(g[1], z) and torch.equal(g[2], v) and g[3] == T + 1
    b2.close()
    bt.close()
