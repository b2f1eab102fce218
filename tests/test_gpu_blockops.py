"""GPU tests of the standalone block operations of the C ABI against the
oracle: inverse quantization, Theorem 1's exact decode of matvec rows, the
encrypted matvec of Eq. (itq2) on one block, and the host checkpoint of the
ADMM object."""
from fractions import Fraction

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


def test_dequantize_inverts_both_quantizers_exactly(env):
    torch, pc2, ctx = env
    rng = np.random.default_rng(1)
    u = np.concatenate([rng.uniform(-8, 8, 997), [-8.0, 8.0, 0.0]])
    du = torch.from_numpy(u).cuda()
    for gamma, oq in ((2, O.gamma2), (1, O.gamma1)):
        q = pc2.quantize(ctx, du, QP.zmin, QP.zmax, QP.log2_scale, gamma)
        back = pc2.dequantize(ctx, q, QP.zmin, QP.log2_scale, gamma).cpu().numpy()
        ref = oq(u, QP)
        assert np.array_equal(q.cpu().numpy(), ref)
        s = 2 ** (QP.log2_scale * (2 if gamma == 1 else 1))
        want = np.array([float(Fraction(int(x), s) + Fraction(QP.zmin)) for x in ref])
        assert np.array_equal(back, want)
        assert np.max(np.abs(back - u)) <= 0.5 / s + 1e-15
    assert ctx.status() == 0


def test_decode_matvec_equals_oracle_decode(env):
    torch, pc2, ctx = env
    rng = np.random.default_rng(2)
    n, limbs = 70, 8
    # magnitudes where the exact sum stays inside 64 bits, as decrypted rows do
    D = [int(x) for x in rng.integers(0, 1 << 60, n)]
    brow = rng.integers(0, 1 << 30, n)
    asum = rng.integers(0, 1 << 33, n).astype(np.uint64)
    nk = rng.integers(1, 8, n).astype(np.int32)
    want = np.array([O.decode([D[i]], [int(brow[i])], int(asum[i]), int(nk[i]), QP)[0] for i in range(n)])
    dD = pc2.ints_to_tiled(ctx, D, limbs)
    x = pc2.decode_matvec(ctx, dD, limbs, n, torch.from_numpy(brow).cuda(), torch.from_numpy(asum.view(np.int64)).cuda(),
                          torch.from_numpy(nk).cuda(), QP.zmin, QP.log2_scale)
    assert np.array_equal(x.cpu().numpy(), want)
    assert ctx.status() == 0


@pytest.mark.parametrize("nbits,n,kbits", [(512, 37, 12), (1024, 70, 28), (2048, 20, 5), (4096, 6, 5)])
def test_hom_matvec_block_equals_oracle(env, nbits, n, kbits):
    torch, pc2, ctx = env
    p, q = W.primes(nbits, 4)
    kg, ko = pc2.Key.from_primes(p, q), P.derive_key(p, q)
    rng = np.random.default_rng(nbits + n)
    a = W.plaintexts_u64(n, seed=3)
    s = W.plaintexts_u64(n, seed=4)
    ah = pc2.encrypt(ctx, kg, torch.from_numpy(a.view(np.int64)).cuda(), 9, 1)
    sh = pc2.encrypt(ctx, kg, torch.from_numpy(s.view(np.int64)).cuda(), 9, 2)
    K = rng.integers(0, 1 << kbits, size=(n, n), dtype=np.uint64)
    dK = torch.from_numpy(K.astype(np.uint32).view(np.int32)).cuda()
    out = pc2.hom_matvec(ctx, kg, ah, sh, dK, n, kbits)
    L2 = 2 * kg.limbs
    got = pc2.tiled_to_ints(ctx, out, n, L2)
    want = P.hom_matvec(ko, pc2.tiled_to_ints(ctx, ah, n, L2), pc2.tiled_to_ints(ctx, sh, n, L2), K)
    assert got == want
    # and the plaintext it carries: a_i + sum_j K_ij s_j mod n
    dec = pc2.tiled_to_ints(ctx, pc2.decrypt(ctx, kg, out, n), n, kg.limbs)
    for i in (0, n - 1):
        assert dec[i] == (int(a[i]) + sum(int(K[i, j]) * int(s[j]) for j in range(n))) % ko.n


def test_admm_host_checkpoint_round_trip(env):
    torch, pc2, ctx = env
    L = W.lasso_small(seed=7, M=30, N=48, nnz=4, K=2)
    st = O.dis_setup(L.A, L.y, W.node_sizes(48, 2), L.rho)
    p, q = W.primes(512, 5)
    kg = pc2.Key.from_primes(p, q)
    alpha = torch.from_numpy(np.concatenate(st.alpha)).cuda()
    Bbar = torch.from_numpy(np.concatenate([b.ravel() for b in st.Bbar])).cuda()

    def make():
        return pc2.Admm(ctx, kg, st.sizes, alpha, Bbar, L.lam, L.rho, QP.zmin, QP.zmax, QP.log2_scale, 13)

    a = make()
    a.round(2)
    x, z, v, r = a.save()
    assert r == 3
    a.round(2)
    b = make()
    b.load(x, z, v, r)
    b.round(2)
    for u, w in zip(a.get()[:3], b.get()[:3]):
        assert torch.equal(u, w)
    ref = O.quantized_admm(st, L.lam, L.rho, 4, QP)
    assert np.array_equal(b.get()[2].cpu().numpy(), ref.v[3])


def test_zv_update_equals_oracle(env):
    """Eqs. (ty32), (u78) elementwise, bit-exact against the oracle's update,
    with v + x landing exactly on +-kappa, on 0 and inside the dead zone."""
    torch, pc2, ctx = env
    rng = np.random.default_rng(3)
    n, kappa = 1000, 0.01
    x = rng.standard_normal(n) * 0.02
    v = rng.standard_normal(n) * 0.02
    x[:4] = [kappa, -kappa, 0.0, 0.004]
    v[:4] = 0.0
    z = rng.standard_normal(n)
    z_ref = O.soft_threshold(v + x, kappa)
    v_ref = v + x - z_ref
    dx, dz, dv = (torch.from_numpy(a.copy()).cuda() for a in (x, z, v))
    pc2.zv_update(ctx, dx, dz, dv, kappa)
    assert np.array_equal(dz.cpu().numpy(), z_ref) and np.array_equal(dv.cpu().numpy(), v_ref)


def test_zv_update_edges_all_magnitudes(env):
    """Eqs. (ty32), (u78) at the threshold's edges and far from them: |v + x|
    at kappa, just above it, at 1.5 and 2 kappa and next to 2 kappa, far
    beyond (where z = v + x - kappa rounds back to v + x), subnormal,
    infinite and NaN sums, both signs, for kappa 0, subnormal, 1, near the
    largest double, and log-uniform magnitudes over the whole double range;
    bit-exact against the oracle (NaN as NaN)."""
    torch, pc2, ctx = env
    rng = np.random.default_rng(5)
    tiny = np.nextafter(0.0, 1.0)
    for kappa in (0.01, 0.0, 1.0, 5 * tiny, 1.2e308, 3.0e-308):
        k2 = 2 * kappa
        eps = np.finfo(np.float64).eps
        pts = [kappa, np.nextafter(kappa, np.inf), 1.5 * kappa, k2, np.nextafter(k2, np.inf), np.nextafter(k2, 0.0),
               3 * kappa, kappa * 2.0 ** 52, kappa * 2.0 ** 53, kappa * 2.0 ** 60, kappa * (1 + eps), 1e300,
               np.finfo(np.float64).max, tiny, 2.2250738585072014e-308, 0.0, np.inf, np.nan, 1.0, 1e-300]
        pts = np.array([p for p in pts if np.isfinite(p) or np.isinf(p) or np.isnan(p)], dtype=np.float64)
        mags = 10.0 ** rng.uniform(-320, 308, 4000)
        x = np.concatenate([pts, -pts, mags * rng.choice([-1.0, 1.0], mags.size)])
        v = np.zeros_like(x)
        v[len(pts) * 2:] = rng.standard_normal(mags.size) * np.where(rng.random(mags.size) < 0.5, kappa, 1.0)
        with np.errstate(invalid="ignore", over="ignore"):
            z_ref = O.soft_threshold(v + x, kappa)
            v_ref = v + x - z_ref
        dx, dz, dv = (torch.from_numpy(a.copy()).cuda() for a in (x, np.full(x.size, 7.0), v))
        pc2.zv_update(ctx, dx, dz, dv, kappa)
        gz, gv = dz.cpu().numpy(), dv.cpu().numpy()
        assert np.array_equal(gz.view(np.int64)[~np.isnan(z_ref)], z_ref.view(np.int64)[~np.isnan(z_ref)]), kappa
        assert np.array_equal(np.isnan(gz), np.isnan(z_ref)), kappa
        ok = ~np.isnan(v_ref)
        assert np.array_equal(gv.view(np.int64)[ok], v_ref.view(np.int64)[ok]), kappa
        assert np.array_equal(np.isnan(gv), np.isnan(v_ref)), kappa


def test_quantize_ties_edges_and_flags(env):
    """Eq. (et21) at exact half-way points (round half to even), at the range
    ends and just inside them, for both quantizers, against the oracle; and the
    clamp and flag for values outside the range, infinities and NaN."""
    torch, pc2, ctx = env
    k = QP.log2_scale
    ties2 = [QP.zmin + (2 * j + 1) * 2.0 ** -(k + 1) for j in range(0, 4000, 7)]
    ties1 = [QP.zmin + (2 * j + 1) * 2.0 ** -(2 * k + 1) for j in range(0, 4000, 7)]
    for gamma, oq, vals in ((2, O.gamma2, ties2), (1, O.gamma1, ties1)):
        half = 0.5 * 2.0 ** -(k if gamma == 2 else 2 * k)      # half a step of this quantizer
        edges = [QP.zmin, QP.zmax, QP.zmin + 2.0 ** -60, QP.zmax - 2.0 ** -40, QP.zmin - half, 0.0, -0.0]
        u = np.array(vals + edges)
        q = pc2.quantize(ctx, torch.from_numpy(u).cuda(), QP.zmin, QP.zmax, k, gamma)
        assert np.array_equal(q.cpu().numpy(), oq(u, QP)), gamma
    assert ctx.status() == 0
    bad = np.array([QP.zmax + 1.0, QP.zmin - 1.0, np.inf, -np.inf, np.nan, 1e300])
    q = pc2.quantize(ctx, torch.from_numpy(bad).cuda(), QP.zmin, QP.zmax, k, 2).cpu().numpy()
    delta = int(round((QP.zmax - QP.zmin) * 2 ** k))
    assert q.tolist() == [delta, 0, delta, 0, 0, delta]
    assert ctx.status() & pc2.ST_QUANT
