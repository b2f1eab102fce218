"""Full-scale private ADMM on the GPU against the oracle: the 256 x 256
image-like LASSO (N = 65536, 16 edge nodes of 4096, A of N/4 x N), 3072-bit
n, lambda 0.005, rho 1 -- two rounds of Algorithm 1 in the batched launch
configuration (round 1 eager, round 2 from the captured CUDA graph).

Every element is checked: x, z, v bit-identical and every decrypted integer
D_i = c_i + sum_j b_ij a_j equal to the oracle's exact value (Eq. (ret54),
65536 rows of 4096 terms); ciphertexts are sampled (z-hat, (-v)-hat on a few
elements, x-hat of one row recomputed by the oracle's Eq. (itq2))."""
import numpy as np
import pytest

from oracle import admm as O
from oracle import paillier as P
from paper_2601_14980_b300 import workloads as W

pytestmark = pytest.mark.gpu

QP = O.QParams(zmin=-8.0, zmax=8.0, log2_scale=24)
SEED = 5


def test_full_scale_3072_bit_rounds_bit_exact():
    import torch

    from paper_2601_14980_b300 import pc2

    ctx = pc2.Context(0)
    x0, sizes, A, y = W.lasso_large_data(device="cuda")
    lam, rho, T = 0.005, 1.0, 2
    # edge-node initialization of Sec. II (input preparation): B_k, alpha_k, Bbar_k
    alphas, bbars = [], []
    for Ak in A:
        n = Ak.shape[1]
        B = torch.linalg.inv(Ak.T @ Ak + rho * torch.eye(n, dtype=torch.float64, device="cuda"))
        alphas.append(B @ (Ak.T @ y))
        bbars.append(rho * B)
    del A
    alpha = torch.cat(alphas)
    Bbar = torch.cat([b.reshape(-1) for b in bbars])
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(int).tolist()
    st = O.DisSetup(sizes=sizes, offsets=offs, B=None, alpha=[a.cpu().numpy() for a in alphas],
                    Bbar=[b.cpu().numpy() for b in bbars])
    del alphas, bbars
    p, q = W.primes(3072, 1)
    kg, ko = pc2.Key.from_primes(p, q), P.derive_key(p, q)
    adm = pc2.Admm(ctx, kg, sizes, alpha, Bbar, lam, rho, QP.zmin, QP.zmax, QP.log2_scale, SEED)
    ref = O.quantized_admm(st, lam, rho, T, QP)
    N, L2 = offs[-1], 2 * kg.limbs
    for t in range(T):
        adm.round(1)
        x, z, v, nxt = adm.get()
        assert nxt == t + 2
        assert np.array_equal(x.cpu().numpy(), ref.x[t]), t
        assert np.array_equal(z.cpu().numpy(), ref.z[t]), t
        assert np.array_equal(v.cpu().numpy(), ref.v[t]), t
    assert ctx.status() == 0
    b = adm.buffers()
    D = pc2.tiled_to_ints(ctx, pc2.device_words(b["D"], pc2.tiled_words(N, kg.limbs)), N, kg.limbs)
    assert D == ref.D[T - 1]
    # ciphertexts of round T, sampled
    zq, vq = O.gamma2(ref.z[T - 2], QP), O.gamma2(-ref.v[T - 2], QP)
    zh = pc2.tiled_to_ints(ctx, pc2.device_words(b["zhat"], pc2.tiled_words(N, L2)), N, L2)
    vh = pc2.tiled_to_ints(ctx, pc2.device_words(b["vhat"], pc2.tiled_words(N, L2)), N, L2)
    for e in (0, 4095, 40000, N - 1):
        assert zh[e] == P.encrypt(ko, [int(zq[e])], [P.r_of(ko, SEED, O.stream_id(T, O.KIND_Z), e)])[0]
        assert vh[e] == P.encrypt(ko, [int(vq[e])], [P.r_of(ko, SEED, O.stream_id(T, O.KIND_V), e)])[0]
    xh = pc2.tiled_to_ints(ctx, pc2.device_words(b["xhat"], pc2.tiled_words(N, L2)), N, L2)
    ah = pc2.tiled_to_ints(ctx, pc2.device_words(b["alpha_hat"], pc2.tiled_words(N, L2)), N, L2)
    k, i = 9, offs[9] + 1234
    o = offs[k]
    s = P.hom_add(ko, zh[o:o + sizes[k]], vh[o:o + sizes[k]])
    row = O.gamma2(st.Bbar[k][i - o:i - o + 1], QP).astype(np.uint64)
    assert xh[i] == P.hom_matvec(ko, [ah[i]], s, row)[0]
    assert P.decrypt(ko, [xh[i]])[0] == ref.D[T - 1][i]
    adm.close()
