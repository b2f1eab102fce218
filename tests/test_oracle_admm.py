"""Pins for the oracle's FP64 ADMM, quantizer, decode and private loop
(oracle/admm.py).

Ties: soft-threshold closed form; the LASSO closed form S_lambda(A^T y) for an
orthonormal design; the KKT conditions of the LASSO at convergence (global for
the centralised ADMM, per block for the distributed one, whose fixed point
solves each node's own LASSO); K = 1 reduces to the centralised ADMM; the
quantizers against their definition; the decode against exact rational
arithmetic; Theorem 1 (real encryption gives the same decrypted integers and
iterates as the plain-integer evaluation); and the quantization error bound."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import admm as O
from oracle import paillier as P
from paper_2601_14980_b300 import workloads as W


def test_soft_threshold_closed_form():
    a = np.array([-3.0, -1.0, -0.5, 0.0, 0.5, 1.0, 1.0000001, 3.0])
    k = 1.0
    expect = np.array([-2.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0000001 - 1.0, 2.0])
    assert np.array_equal(O.soft_threshold(a, k), expect)


def test_cen_admm_orthonormal_design_closed_form():
    rng = np.random.default_rng(0)
    M, N = 60, 40
    A, _ = np.linalg.qr(rng.standard_normal((M, N)))   # A^T A = I
    y = rng.standard_normal(M)
    lam, rho = 0.3, 1.0
    x, z, v = O.cen_admm(A, y, lam, rho, 400)
    xstar = O.soft_threshold(A.T @ y, lam)
    assert np.allclose(z, xstar, atol=1e-10)


def _kkt_gap(A, y, x, lam):
    g = A.T @ (y - A @ x)
    nz = np.abs(x) > 1e-9
    gap_nz = np.max(np.abs(g[nz] - lam * np.sign(x[nz]))) if nz.any() else 0.0
    gap_z = np.max(np.abs(g[~nz]) - lam) if (~nz).any() else -1.0
    return gap_nz, gap_z


def test_cen_admm_kkt():
    L = W.lasso_small(seed=5, M=40, N=80, nnz=6)
    x, z, v = O.cen_admm(L.A, L.y, 0.05, 1.0, 3000)
    gnz, gz = _kkt_gap(L.A, L.y, z, 0.05)
    assert gnz < 1e-6 and gz < 1e-6


def test_dis_admm_blockwise_kkt_and_k1():
    L = W.lasso_small(seed=6, M=40, N=80, nnz=6)
    sizes = W.node_sizes(80, 4)
    st = O.dis_setup(L.A, L.y, sizes, 1.0)
    x, z, v = O.dis_admm(st, 0.05, 1.0, 3000)
    for a0, a1 in zip(st.offsets[:-1], st.offsets[1:]):
        gnz, gz = _kkt_gap(L.A[:, a0:a1], L.y, z[a0:a1], 0.05)
        assert gnz < 1e-6 and gz < 1e-6
    st1 = O.dis_setup(L.A, L.y, [80], 1.0)
    xd, zd, vd = O.dis_admm(st1, 0.05, 1.0, 7)
    xc, zc, vc = O.cen_admm(L.A, L.y, 0.05, 1.0, 7)
    assert np.allclose(xd, xc, rtol=1e-11, atol=1e-12) and np.allclose(zd, zc, rtol=1e-11, atol=1e-12)


def test_jacobi_schedule_reading():
    # Eq. (loi32) taken literally (z^t, v^t from x^{t-1}) starting from zeros:
    # round 1 leaves z = v = 0, and round 2 then performs the first
    # Gauss-Seidel z/v update, so z_J^2 = z_GS^1 and v_J^2 = v_GS^1.
    L = W.lasso_small(seed=7, M=30, N=40, nnz=4)
    st = O.dis_setup(L.A, L.y, W.node_sizes(40, 2), 1.0)
    x1, z1, v1 = O.dis_admm(st, 0.02, 1.0, 1, jacobi=True)
    assert not z1.any() and not v1.any()
    _, zj, vj = O.dis_admm(st, 0.02, 1.0, 2, jacobi=True)
    xg, zg, vg = O.dis_admm(st, 0.02, 1.0, 1)
    assert np.array_equal(x1, xg) and np.array_equal(zj, zg) and np.array_equal(vj, vg)


def test_quantizers_definition():
    qp = O.QParams(zmin=-8.0, zmax=8.0, log2_scale=24)
    S = 2 ** 24
    u = np.array([-8.0, 8.0, 0.0, -7.999999, 1.5, 0.1])
    q2 = O.gamma2(u, qp)
    for ui, qi in zip(u, q2):
        exact = (Fraction(float(ui)) - Fraction(-8)) * S
        assert abs(Fraction(int(qi)) - exact) <= Fraction(1, 2)
    assert q2[0] == 0 and q2[1] == qp.delta
    # ties round to even: (u - zmin) * S = k + 1/2 exactly
    tie = -8.0 + (5 + 0.5) / S
    assert O.gamma2(np.array([tie]), qp)[0] == 6
    tie2 = -8.0 + (6 + 0.5) / S
    assert O.gamma2(np.array([tie2]), qp)[0] == 6
    q1 = O.gamma1(np.array([0.25]), qp)
    assert q1[0] == int((Fraction(0.25) + 8) * S * S)
    with pytest.raises(ValueError):
        O.gamma2(np.array([8.5]), qp)


def test_decode_equals_exact_rational():
    # x_i must be the float64 rounding of alpha~_i + sum_j B~_ij w~_j computed
    # exactly from the dequantized inputs.
    qp = O.QParams(zmin=-8.0, zmax=8.0, log2_scale=24)
    rng = np.random.default_rng(3)
    Nk = 7
    alpha = rng.standard_normal(Nk)
    Bbar = rng.standard_normal((Nk, Nk)) * 0.3
    z = rng.standard_normal(Nk)
    v = rng.standard_normal(Nk)
    c = O.gamma1(alpha, qp)
    b = O.gamma2(Bbar, qp)
    zq, vq = O.gamma2(z, qp), O.gamma2(-v, qp)
    a = [int(x) + int(y) for x, y in zip(zq, vq)]
    D = [int(c[i]) + sum(int(b[i, j]) * a[j] for j in range(Nk)) for i in range(Nk)]
    x = O.decode(D, [int(s) for s in b.sum(axis=1)], sum(a), Nk, qp)
    S = Fraction(2 ** 24)
    for i in range(Nk):
        at = Fraction(int(c[i])) / (S * S) + Fraction(-8)
        val = at + sum((Fraction(int(b[i, j])) / S + Fraction(-8)) * (Fraction(a[j]) / S + 2 * Fraction(-8)) for j in range(Nk))
        assert x[i] == float(val)


def _setup_tiny(seed=11, N=12, K=2, M=10):
    L = W.lasso_small(seed=seed, M=M, N=N, nnz=3, K=K)
    st = O.dis_setup(L.A, L.y, W.node_sizes(N, K), 1.0)
    return L, st


def test_theorem1_private_equals_quantized():
    L, st = _setup_tiny()
    qp = O.QParams(zmin=-8.0, zmax=8.0, log2_scale=24)
    p, q = W.primes(256, 9)
    key = P.derive_key(p, q)
    pr = O.private_admm(st, 0.01, 1.0, 3, qp, key, seed=1234)
    qz = O.quantized_admm(st, 0.01, 1.0, 3, qp)
    for t in range(3):
        assert pr.D[t] == qz.D[t]
        assert np.array_equal(pr.x[t], qz.x[t])
        assert np.array_equal(pr.z[t], qz.z[t]) and np.array_equal(pr.v[t], qz.v[t])
        assert max(pr.D[t]) < key.n


def test_quantization_error_bound_and_mse():
    L, st = _setup_tiny(seed=12, N=24, K=3, M=16)
    qp = O.QParams(zmin=-8.0, zmax=8.0, log2_scale=24)
    T = 6
    qz = O.quantized_admm(st, 0.01, 1.0, T, qp)
    # plain Dis-ADMM trajectory
    xs = []
    for t in range(1, T + 1):
        x, _, _ = O.dis_admm(st, 0.01, 1.0, t)
        xs.append(x)
    # round 1: same (z, v) = 0 input
    eps1 = O.round_error_bound(st, qp, np.zeros(24), np.zeros(24), qz.x[0])
    assert np.all(np.abs(qz.x[0] - xs[0]) <= eps1 + 1e-14)
    # whole run: G_t <= 2 G_{t-1} + ||eps_t||, ||x_priv^T - x_plain^T|| <= G_{T-1} + ||eps_T||
    G = 0.0
    zp, vp = np.zeros(24), np.zeros(24)
    for t in range(T):
        e = np.linalg.norm(O.round_error_bound(st, qp, zp, vp, qz.x[t]))
        bound_t = G + e
        assert np.linalg.norm(qz.x[t] - xs[t]) <= bound_t + 1e-12
        G = 2 * G + e
        zp, vp = qz.z[t], qz.v[t]
    dT = bound_t + 1e-12
    mse_priv = np.mean((qz.x[-1] - L.x0) ** 2)
    mse_plain = np.mean((xs[-1] - L.x0) ** 2)
    assert abs(mse_priv - mse_plain) <= (2 * np.linalg.norm(xs[-1] - L.x0) * dT + dT ** 2) / 24
    # the Douglas-Rachford bound (linear in the rounds) holds too, and is tighter
    d2, mb = O.mse_gap_bound(st, qp, qz.x, qz.z, qz.v, xs[-1], L.x0)
    assert np.linalg.norm(qz.x[-1] - xs[-1]) <= d2 < dT
    assert abs(mse_priv - mse_plain) <= mb
    for t in range(1, T + 1):   # every prefix of the run
        dt, _ = O.mse_gap_bound(st, qp, qz.x[:t], qz.z[:t], qz.v[:t], xs[t - 1], L.x0)
        assert np.linalg.norm(qz.x[t - 1] - xs[t - 1]) <= dt


def test_diag_setup_is_the_orthonormal_closed_form():
    """diag_setup equals the general initialization (B_k = (A_k^T A_k + rho I)^-1)
    for an orthonormal design, and its Dis-ADMM reaches the LASSO closed form."""
    rng = np.random.default_rng(3)
    M, sizes, rho, lam = 80, [7, 20, 13], 1.0, 0.05
    N = sum(sizes)
    A, _ = np.linalg.qr(rng.standard_normal((M, N)))
    y = rng.standard_normal(M)
    full = O.dis_setup(A, y, sizes, rho)
    diag = O.diag_setup(A.T @ y, rho)
    alpha_full = np.concatenate(full.alpha)
    alpha_diag = np.array([a[0] for a in diag.alpha])
    assert np.allclose(alpha_full, alpha_diag, atol=1e-14)
    for k, Bb in enumerate(full.Bbar):
        o = full.offsets[k]
        assert np.allclose(Bb, np.diag([diag.Bbar[o + i][0, 0] for i in range(sizes[k])]), atol=1e-14)
    x, z, v = O.dis_admm(diag, lam, rho, 300)
    assert np.allclose(z, O.soft_threshold(A.T @ y, lam), atol=1e-9)


def test_one_by_one_blocks_equal_diagonal_node_blocks_exactly():
    """With a diagonal Bbar_k the quantized round over N_k x N_k node blocks and
    over 1 x 1 blocks give identical iterates: the off-diagonal b_ij = Gamma2(0)
    dequantize to exactly zero in the exact decode."""
    rng = np.random.default_rng(4)
    sizes, rho, lam = [5, 9, 4], 1.0, 0.02
    aty = rng.standard_normal(sum(sizes))
    qp = O.QParams(zmin=-8.0, zmax=8.0, log2_scale=24)
    diag = O.diag_setup(aty, rho)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(int).tolist()
    blocks = O.DisSetup(sizes=sizes, offsets=offs,
                        B=[np.eye(n) / (1 + rho) for n in sizes],
                        alpha=[np.array([diag.alpha[i][0] for i in range(offs[k], offs[k + 1])])
                               for k in range(len(sizes))],
                        Bbar=[np.diag([diag.Bbar[i][0, 0] for i in range(offs[k], offs[k + 1])])
                              for k in range(len(sizes))])
    a = O.quantized_admm(diag, lam, rho, 4, qp)
    b = O.quantized_admm(blocks, lam, rho, 4, qp)
    for t in range(4):
        assert np.array_equal(a.x[t], b.x[t]) and np.array_equal(a.z[t], b.z[t]) and np.array_equal(a.v[t], b.v[t])


def test_batch_problem_shape():
    bp = W.batch_problem(seed=1, nodes=10, lo=8, hi=100)
    assert len(bp.sizes) == 10 and all(8 <= s <= 100 for s in bp.sizes)
    assert len(bp.aty) == sum(bp.sizes) and bp.node_key[:4] == [0, 1, 2, 0]


def test_exact_rowdot_split_equals_python_integers():
    """The int64 split of exact_rowdot against term-by-term Python integers,
    including the largest operands the quantizer produces (b = Delta, a = 2 Delta)."""
    rng = np.random.default_rng(7)
    delta = 16 << 24
    b = rng.integers(0, delta + 1, size=(300, 400), dtype=np.int64)
    b[0, :] = delta
    a = [int(x) for x in rng.integers(0, 2 * delta + 1, size=400)]
    a[:5] = [2 * delta] * 5
    want = [sum(int(b[i, j]) * a[j] for j in range(400)) for i in range(300)]
    assert O.exact_rowdot(b, a) == want        # split path (b.size > 2^16)
    small = b[:100, :50]
    assert O.exact_rowdot(small, a[:50]) == [sum(int(small[i, j]) * a[j] for j in range(50)) for i in range(100)]


def test_precision_loss_falls_as_one_over_delta():
    # The paper's experiment on the quantization's precision loss (a 3 x 3
    # design, Delta swept over many decades): the private iterate differs from
    # plaintext Dis-ADMM by O(1/Delta).  Here Delta = S (zmax - zmin) with
    # S = 2^8 .. 2^28 (the Gamma1 scale S^2 Delta must stay below 2^63), 20
    # rounds; the gap shrinks with every step of S and stays within a fixed
    # multiple of 1/Delta.
    L = W.lasso_small(seed=2, M=3, N=3, nnz=1, K=3, lam=0.01, rho=1.0)
    st = O.dis_setup(L.A, L.y, W.node_sizes(3, 3), L.rho)
    xp = O.dis_admm(st, L.lam, L.rho, 20)[0]
    gaps = []
    for k in (8, 12, 16, 20, 24, 28):
        qp = O.QParams(zmin=-8.0, zmax=8.0, log2_scale=k)
        gap = float(np.max(np.abs(O.quantized_admm(st, L.lam, L.rho, 20, qp).x[-1] - xp)))
        delta = 16.0 * 2.0 ** k
        assert 0.5 <= gap * delta <= 64.0, (k, gap * delta)
        gaps.append(gap)
    assert all(b < a for a, b in zip(gaps, gaps[1:]))


def test_douglas_rachford_bound_coarse_quantizer_many_rounds():
    """With a coarse scale (S = 2^8) the quantization errors are large and the
    bound is tested where it is nearly tight: for 40 rounds the private
    iterate stays within Delta_t of plaintext Dis-ADMM at every round."""
    L, st = _setup_tiny(seed=13, N=24, K=3, M=16)
    qp = O.QParams(zmin=-8.0, zmax=8.0, log2_scale=8)
    T = 40
    qz = O.quantized_admm(st, 0.01, 1.0, T, qp)
    ratios = []
    for t in range(1, T + 1):
        x_plain, _, _ = O.dis_admm(st, 0.01, 1.0, t)
        dt, mb = O.mse_gap_bound(st, qp, qz.x[:t], qz.z[:t], qz.v[:t], x_plain, L.x0)
        gap = np.linalg.norm(qz.x[t - 1] - x_plain)
        assert gap <= dt, t
        assert abs(np.mean((qz.x[t - 1] - L.x0) ** 2) - np.mean((x_plain - L.x0) ** 2)) <= mb
        ratios.append(gap / dt)
    assert max(ratios) > 1e-3      # the bound is not vacuous at this scale
