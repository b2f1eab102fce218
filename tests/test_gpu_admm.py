"""GPU parity of the private ADMM round (Algorithm 1) against the oracle.

Setup integers come from the same FP64 set-up (oracle.admm.dis_setup) on both
sides, so the decrypted integers, the exact decode and therefore every
iterate are bit-identical; ciphertexts are bit-identical given the same
Philox draws.  The plaintext Dis-ADMM path differs only in summation order
(relative 1e-9)."""
import numpy as np
import pytest

from oracle import admm as O
from oracle import paillier as P
from paper_2601_14980_b300 import workloads as W

pytestmark = pytest.mark.gpu

QP = O.QParams(zmin=-8.0, zmax=8.0, log2_scale=24)


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2601_14980_b300 import pc2

    return torch, pc2, pc2.Context(0)


def _make(env, L, nbits, seed=1, per_node=False, key_seed=1):
    torch, pc2, ctx = env
    st = O.dis_setup(L.A, L.y, W.node_sizes(L.A.shape[1], L.K), L.rho)
    p, q = W.primes(nbits, key_seed)
    kg, ko = pc2.Key.from_primes(p, q), P.derive_key(p, q)
    alpha = torch.from_numpy(np.concatenate(st.alpha)).cuda()
    Bbar = torch.from_numpy(np.concatenate([b.ravel() for b in st.Bbar])).cuda()
    adm = pc2.Admm(ctx, kg, st.sizes, alpha, Bbar, L.lam, L.rho, QP.zmin, QP.zmax, QP.log2_scale, seed,
                   per_node=per_node)
    return st, kg, ko, adm


def _ints(pc2, ptr, count, limbs):
    w = pc2.device_words(ptr, pc2.tiled_words(count, limbs))
    return w


def test_private_rounds_match_oracle_bit_exact(env):
    torch, pc2, ctx = env
    L = W.lasso_small(seed=1)                  # 128 x 256, 4 nodes, lambda 0.01, rho 1, 5 rounds
    st, kg, ko, adm = _make(env, L, 1024)
    ref = O.quantized_admm(st, L.lam, L.rho, L.iters, QP)
    for t in range(L.iters):
        adm.round(1)                           # round 1 eager, later rounds replay the CUDA graph
        x, z, v, nxt = adm.get()
        assert nxt == t + 2
        assert np.array_equal(x.cpu().numpy(), ref.x[t]), t
        assert np.array_equal(z.cpu().numpy(), ref.z[t]), t
        assert np.array_equal(v.cpu().numpy(), ref.v[t]), t
        b = adm.buffers()
        D = pc2.tiled_to_ints(ctx, _ints(pc2, b["D"], 256, kg.limbs), 256, kg.limbs)
        assert D == ref.D[t], t
    assert ctx.status() == 0
    # ciphertexts of the last round, sampled: z-hat, (-v)-hat and x-hat rows
    T = L.iters
    zprev = ref.z[T - 2] if T > 1 else np.zeros(256)
    vprev = ref.v[T - 2] if T > 1 else np.zeros(256)
    zq, vq = O.gamma2(zprev, QP), O.gamma2(-vprev, QP)
    b = adm.buffers()
    zh = pc2.tiled_to_ints(ctx, _ints(pc2, b["zhat"], 256, 2 * kg.limbs), 256, 2 * kg.limbs)
    vh = pc2.tiled_to_ints(ctx, _ints(pc2, b["vhat"], 256, 2 * kg.limbs), 256, 2 * kg.limbs)
    xh = pc2.tiled_to_ints(ctx, _ints(pc2, b["xhat"], 256, 2 * kg.limbs), 256, 2 * kg.limbs)
    ah = pc2.tiled_to_ints(ctx, _ints(pc2, b["alpha_hat"], 256, 2 * kg.limbs), 256, 2 * kg.limbs)
    for e in (0, 63, 64, 200, 255):
        assert zh[e] == P.encrypt(ko, [int(zq[e])], [P.r_of(ko, 1, O.stream_id(T, O.KIND_Z), e)])[0]
        assert vh[e] == P.encrypt(ko, [int(vq[e])], [P.r_of(ko, 1, O.stream_id(T, O.KIND_V), e)])[0]
    # x-hat rows 0 and 130 recomputed by the oracle's Eq. (itq2) from the GPU's own alpha-hat, s-hat
    bq = [O.gamma2(B, QP) for B in st.Bbar]
    s = P.hom_add(ko, zh, vh)
    for i in (0, 130):
        k, o = i // 64, (i // 64) * 64
        row = bq[k][i - o:i - o + 1].astype(np.uint64)
        assert xh[i] == P.hom_matvec(ko, [ah[i]], s[o:o + 64], row)[0]


def test_final_mse_within_quantization_bound(env):
    """The small LASSO's five private GPU rounds end within the stated
    quantization bound of plaintext Dis-ADMM (Theorem 1's errors carried
    through the rounds): |MSE_priv - MSE_plain| <= bound, with the bound
    computed from the GPU's own iterates and the plaintext path on the GPU."""
    torch, pc2, ctx = env
    L = W.lasso_small(seed=1)
    st, kg, ko, adm = _make(env, L, 1024)
    xs, zs, vs = [], [], []
    for t in range(L.iters):
        adm.round(1)
        x, z, v, _ = adm.get()
        xs.append(x.cpu().numpy()), zs.append(z.cpu().numpy()), vs.append(v.cpu().numpy())
    adm.reset()
    adm.round_plain(L.iters)
    x_plain = adm.get()[0].cpu().numpy()
    dT, bound = O.mse_gap_bound(st, QP, xs, zs, vs, x_plain, L.x0)
    mse_priv = float(np.mean((xs[-1] - L.x0) ** 2))
    mse_plain = float(np.mean((x_plain - L.x0) ** 2))
    assert np.linalg.norm(xs[-1] - x_plain) <= dT
    assert abs(mse_priv - mse_plain) <= bound
    assert ctx.status() == 0


def test_tiny_problem_against_real_encryption_oracle(env):
    torch, pc2, ctx = env
    L = W.lasso_small(seed=11, M=10, N=12, nnz=3, K=2)
    st, kg, ko, adm = _make(env, L, 256, seed=1234, key_seed=9)
    pr = O.private_admm(st, 0.01, 1.0, 3, QP, ko, seed=1234)
    for t in range(3):
        adm.round(1)
        x, z, v, _ = adm.get()
        assert np.array_equal(x.cpu().numpy(), pr.x[t]) and np.array_equal(z.cpu().numpy(), pr.z[t])
        b = adm.buffers()
        for name, ref in (("zhat", pr.zhat[t]), ("vhat", pr.vhat[t]), ("xhat", pr.xhat[t])):
            got = pc2.tiled_to_ints(ctx, _ints(pc2, b[name], 12, 2 * kg.limbs), 12, 2 * kg.limbs)
            assert got == ref, (name, t)


def test_per_node_path_equals_batched(env):
    torch, pc2, ctx = env
    L = W.lasso_small(seed=2, M=64, N=200, nnz=10, K=3)   # uneven nodes 67/67/66, not tile aligned
    _, _, _, a1 = _make(env, L, 512, seed=5)
    _, _, _, a2 = _make(env, L, 512, seed=5, per_node=True)
    a1.round(3)
    a2.round(3)
    for u, w in zip(a1.get()[:3], a2.get()[:3]):
        assert torch.equal(u, w)


def test_plain_dis_admm_and_checkpoint(env):
    torch, pc2, ctx = env
    L = W.lasso_small(seed=3)
    st, kg, ko, adm = _make(env, L, 1024)
    adm.round_plain(7)
    x, z, v, _ = adm.get()
    xr, zr, vr = O.dis_admm(st, L.lam, L.rho, 7)
    np.testing.assert_allclose(x.cpu().numpy(), xr, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(z.cpu().numpy(), zr, rtol=1e-9, atol=1e-12)
    # checkpoint / resume: 2 rounds, save, 3 more on a fresh object == 5 rounds
    adm.reset()
    adm.round(2)
    x2, z2, v2, r2 = adm.get()
    _, _, _, adm_b = _make(env, L, 1024)
    adm_b.set(x2, z2, v2, r2)
    adm_b.round(3)
    adm.round(3)
    for u, w in zip(adm.get()[:3], adm_b.get()[:3]):
        assert torch.equal(u, w)


def test_quantize_entry_point(env):
    torch, pc2, ctx = env
    u = np.array([-8.0, 8.0, 0.0, -7.999999, 1.5, 0.1, -8.0 + 5.5 / 2**24, 3.25])
    du = torch.from_numpy(u).cuda()
    q2 = pc2.quantize(ctx, du, -8.0, 8.0, 24, gamma=2).cpu().numpy()
    assert np.array_equal(q2, O.gamma2(u, QP))
    q1 = pc2.quantize(ctx, du, -8.0, 8.0, 24, gamma=1).cpu().numpy()
    assert np.array_equal(q1, O.gamma1(u, QP))
    qn = pc2.quantize(ctx, du, -8.0, 8.0, 24, gamma=2, negate=True).cpu().numpy()
    assert np.array_equal(qn, O.gamma2(-u, QP))
    assert ctx.status() == 0
    pc2.quantize(ctx, torch.tensor([9.0], dtype=torch.float64, device="cuda"), -8.0, 8.0, 24)
    assert ctx.status() & pc2.ST_QUANT


@pytest.mark.parametrize("nbits,lanes", [(256, 1), (256, 4), (512, 2), (512, 8), (1024, 1), (1024, 4),
                                         (2048, 2), (2048, 8), (3072, 4), (3072, 8), (4096, 4), (4096, 8)])
def test_lanes_per_element_rounds_bit_exact(env, nbits, lanes):
    """Every built lane count of the matvec (and of encryption/decryption where built) gives the oracle's iterates."""
    torch, pc2, ctx = env
    L = W.lasso_small(seed=4, M=24, N=40, nnz=4, K=3)   # nodes 14/13/13: ragged row tiles
    pc2.set_lanes(ctx, lanes)
    try:
        st, kg, ko, adm = _make(env, L, nbits, seed=77)
        ref = O.quantized_admm(st, L.lam, L.rho, 3, QP)
        for t in range(3):
            adm.round(1)
            x, z, v, _ = adm.get()
            assert np.array_equal(x.cpu().numpy(), ref.x[t]), (t, lanes)
            assert np.array_equal(z.cpu().numpy(), ref.z[t]), (t, lanes)
            assert np.array_equal(v.cpu().numpy(), ref.v[t]), (t, lanes)
    finally:
        pc2.set_lanes(ctx, 0)
    assert ctx.status() == 0


@pytest.mark.parametrize("nbits", [512, 2048])
def test_matvec_forms_bit_identical(env, nbits):
    """Rows per CTA and windows spread over CTAs give the same iterates (and the oracle's)."""
    torch, pc2, ctx = env
    L = W.lasso_small(seed=6, M=40, N=90, nnz=5, K=3)      # nodes of 30: ragged row tiles
    ref = None
    for mode in (1, 2):
        st, kg, ko, adm = _make(env, L, nbits, seed=21)
        adm.set_matvec(mode)
        if ref is None:
            ref = O.quantized_admm(st, L.lam, L.rho, 3, QP)
        for t in range(3):
            adm.round(1)
            x, z, v, _ = adm.get()
            assert np.array_equal(x.cpu().numpy(), ref.x[t]), (mode, t)
            assert np.array_equal(v.cpu().numpy(), ref.v[t]), (mode, t)
        adm.close()
    assert ctx.status() == 0


@pytest.mark.parametrize("per_node", [False, True])
def test_tensor_core_engine_rounds_bit_exact(env, per_node):
    """2048-bit n with the engine forced to the tensor cores: the rounds'
    encryptions (z-hat and (-v)-hat in one call, r-streams from the device
    round counter) and decryptions take the tensor-core kernels, inside the
    captured round graph from round 2 on; iterates equal the oracle's."""
    torch, pc2, ctx = env
    L = W.lasso_small(seed=7, M=24, N=60, nnz=4, K=2)
    pc2.set_engine(ctx, pc2.ENGINE_TC)
    try:
        st, kg, ko, adm = _make(env, L, 2048, seed=23, per_node=per_node)
        ref = O.quantized_admm(st, L.lam, L.rho, 3, QP)
        for t in range(3):
            adm.round(1)
            x, z, v, nxt = adm.get()
            assert nxt == t + 2
            assert np.array_equal(x.cpu().numpy(), ref.x[t]) and np.array_equal(v.cpu().numpy(), ref.v[t]), t
        b = adm.buffers()
        D = pc2.tiled_to_ints(ctx, _ints(pc2, b["D"], 60, kg.limbs), 60, kg.limbs)
        assert D == ref.D[2]
        assert ctx.status() == 0
        adm.close()
    finally:
        pc2.set_engine(ctx, -1)


@pytest.mark.parametrize("per_node", [False, True])
def test_missing_edge_node_refuses_round_then_resumes(env, per_node):
    """Failure detection: while an edge node's segment is marked missing the
    round is refused (PC2_EMISSING) with x, z, v and the round counter
    untouched; once it is marked present again the rounds continue and match
    the oracle's iterates bit for bit (batched form, whose rounds replay a
    CUDA graph, and per-node form)."""
    torch, pc2, ctx = env
    L = W.lasso_small(seed=1)
    st, kg, ko, adm = _make(env, L, 1024, per_node=per_node)
    ref = O.quantized_admm(st, L.lam, L.rho, 3, QP)
    adm.round(1)
    x0, z0, v0, r0 = (a.clone() if hasattr(a, "clone") else a for a in adm.get())
    adm.set_node_present(2, False)
    with pytest.raises(pc2.Pc2Error) as err:
        adm.round(1)
    assert err.value.code == pc2.EMISSING
    x1, z1, v1, r1 = adm.get()
    assert r1 == r0 == 2
    assert torch.equal(x1, x0) and torch.equal(z1, z0) and torch.equal(v1, v0)
    with pytest.raises(pc2.Pc2Error):
        adm.set_node_present(L.K, False)      # no such node
    adm.set_node_present(2, True)
    adm.round(2)
    x, z, v, nxt = adm.get()
    assert nxt == 4
    assert np.array_equal(x.cpu().numpy(), ref.x[2]) and np.array_equal(v.cpu().numpy(), ref.v[2])
    assert ctx.status() == 0
