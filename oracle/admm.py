"""FP64 ADMM for the LASSO and the private 3P-ADMM-PC2 loop (CPU oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Follows the paper step by step, in numpy float64 and Python integers:

* ``soft_threshold``  -- S_kappa of Eq. (ty32): a-kappa above kappa, a+kappa
  below -kappa, 0 in between.
* ``cen_admm``        -- Eqs. (sldo09), (ty32), (u78): centralised ADMM.
* ``dis_setup`` / ``dis_admm`` -- column split of Eq. (lop32); local update
  Eq. (sldo091) x_k = B_k (A_k^T y + rho (z_k - v_k)) with
  B_k = (A_k^T A_k + rho I)^{-1}; written as x_k = alpha_k + Bbar_k (z_k - v_k)
  with alpha_k = B_k A_k^T y and Bbar_k = rho B_k (the quantities the
  protocol of Sec. II exchanges).  Default schedule: z and v from this
  round's x (Gauss-Seidel, as Eqs. (sldo09)-(u78)); ``jacobi=True`` takes
  Eq. (loi32) literally (z, v from the previous round's x).
* ``gamma1`` / ``gamma2`` -- quantizers of Eq. (et21) with one public range
  [zmin, zmax] (Theorem 1's reading) and scale S = Delta/(zmax - zmin):
  Gamma2(u) = rint((u - zmin) S), Gamma1(u) = rint((u - zmin) S^2).
* ``decode``          -- inverse quantization of Sec. III-C written out
  exactly (Theorem 1 with the matrix product expanded; see the function).
* ``private_admm``    -- Algorithm 1 with real Paillier encryption
  (oracle.paillier), and ``quantized_admm`` -- the same loop with the
  decrypted integer replaced by the plain integer of Eq. (ret54), which
  Theorem 1 and Paillier correctness say it equals.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

from . import paillier as P

# r-stream ids for the three encrypted vectors of Eq. (itq1)
KIND_ALPHA, KIND_Z, KIND_V = 0, 1, 2


def stream_id(t: int, kind: int) -> int:
    """Philox stream of the r values for vector `kind` in round t (alpha uses t=0)."""
    return (t << 8) | kind


def soft_threshold(a: np.ndarray, kappa: float) -> np.ndarray:
    """S_kappa(a), Eq. (ty32)."""
    a = np.asarray(a, dtype=np.float64)
    out = np.zeros_like(a)
    hi = a > kappa
    lo = a < -kappa
    out[hi] = a[hi] - kappa
    out[lo] = a[lo] + kappa
    return out


def cen_admm(A, y, lam, rho, iters):
    """Centralised ADMM, Eqs. (sldo09), (ty32), (u78)."""
    N = A.shape[1]
    Pinv = np.linalg.inv(A.T @ A + rho * np.eye(N))
    Aty = A.T @ y
    z = np.zeros(N)
    v = np.zeros(N)
    x = np.zeros(N)
    for _ in range(iters):
        x = Pinv @ (Aty + rho * (z - v))
        z = soft_threshold(v + x, lam / rho)
        v = v + x - z
    return x, z, v


@dataclass
class DisSetup:
    sizes: list
    offsets: list
    B: list        # B_k = (A_k^T A_k + rho I)^{-1}
    alpha: list    # alpha_k = B_k A_k^T y
    Bbar: list     # rho B_k


def dis_setup(A, y, sizes, rho) -> DisSetup:
    """Initialization phase of Sec. II: each edge node k forms B_k; the
    master forms alpha_k = B_k A_k^T y."""
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(int).tolist()
    B, alpha, Bbar = [], [], []
    for k in range(len(sizes)):
        Ak = A[:, offs[k]:offs[k + 1]]
        Bk = np.linalg.inv(Ak.T @ Ak + rho * np.eye(sizes[k]))
        B.append(Bk)
        alpha.append(Bk @ (Ak.T @ y))
        Bbar.append(rho * Bk)
    return DisSetup(sizes=list(sizes), offsets=offs, B=B, alpha=alpha, Bbar=Bbar)


def diag_setup(aty, rho) -> DisSetup:
    """Initialization of Sec. II for an orthonormal design (A^T A = I):
    B = (I + rho I)^-1 = I / (1 + rho), alpha = B A^T y, Bbar = rho B, all
    diagonal, written as 1 x 1 blocks (one per element) so that the per-node
    products of Eq. (sldo091) / Eq. (itq2) reduce to their diagonal terms."""
    aty = np.asarray(aty, dtype=np.float64)
    N = len(aty)
    Bk = np.array([[1.0 / (1.0 + rho)]])
    return DisSetup(sizes=[1] * N, offsets=list(range(N + 1)), B=[Bk] * N,
                    alpha=[np.array([a / (1.0 + rho)]) for a in aty], Bbar=[rho * Bk] * N)


def dis_admm(setup: DisSetup, lam, rho, iters, jacobi: bool = False):
    """Distributed (plaintext) ADMM: Eq. (sldo091) per node, then Eqs. (ty32),
    (u78) at the master.  Returns (x, z, v) after `iters` rounds."""
    N = setup.offsets[-1]
    z = np.zeros(N)
    v = np.zeros(N)
    x = np.zeros(N)
    for _ in range(iters):
        xn = np.empty(N)
        for k, (a0, a1) in enumerate(zip(setup.offsets[:-1], setup.offsets[1:])):
            xn[a0:a1] = setup.alpha[k] + setup.Bbar[k] @ (z[a0:a1] - v[a0:a1])
        xu = x if jacobi else xn
        z_new = soft_threshold(v + xu, lam / rho)
        v = v + xu - z_new
        z = z_new
        x = xn
    return x, z, v


# ------------------------------------------------------------------ quantizer


@dataclass(frozen=True)
class QParams:
    """Public quantization range and scale: Delta = S (zmax - zmin).
    zmin * S must be an integer (exact decode)."""

    zmin: float
    zmax: float
    log2_scale: int

    @property
    def S(self) -> float:
        return float(2 ** self.log2_scale)

    @property
    def mS(self) -> int:
        v = self.zmin * self.S
        if v != int(v):
            raise ValueError("zmin * S must be an integer")
        return int(v)

    @property
    def delta(self) -> int:
        return int(round((self.zmax - self.zmin) * self.S))


def gamma2(u, qp: QParams) -> np.ndarray:
    """Gamma2 of Eq. (et21): rint((u - zmin) * S) in {0..Delta} (int64)."""
    u = np.asarray(u, dtype=np.float64)
    t = np.rint((u - qp.zmin) * qp.S)
    if np.any(t < 0) or np.any(t > qp.delta):
        raise ValueError("value outside the public quantization range")
    return t.astype(np.int64)


def gamma1(u, qp: QParams) -> np.ndarray:
    """Gamma1 of Eq. (et21) with scale S^2: rint((u - zmin) * S^2) (int64)."""
    u = np.asarray(u, dtype=np.float64)
    t = np.rint((u - qp.zmin) * (qp.S * qp.S))
    if np.any(t < 0) or np.any(t > float(qp.delta) * qp.S):
        raise ValueError("value outside the public quantization range")
    return t.astype(np.int64)


def dequant2(q, qp: QParams):
    """Inverse of Gamma2 as an exact rational: q/S + zmin."""
    return [Fraction(int(v), 2 ** qp.log2_scale) + Fraction(qp.zmin) for v in np.ravel(q)]


def decode(D: list, brow: list, asum: int, Nk: int, qp: QParams) -> np.ndarray:
    """Inverse quantization of Sec. III-C written out exactly.

    With c = Gamma1(alpha), b = Gamma2(Bbar), a_j = Gamma2(z_j)+Gamma2(-v_j),
    D_i = c_i + sum_j b_ij a_j (the decrypted plaintext), and the dequantized
    values alpha~ = c/S^2 + zmin, B~ = b/S + zmin, w~ = a/S + 2 zmin,

        S^2 (alpha~_i + sum_j B~_ij w~_j)
          = D_i + mS*S + 2 mS sum_j b_ij + mS sum_j a_j + 2 mS^2 N_k,

    with mS = zmin*S.  The right side is an exact integer X_i; the result is
    X_i rounded once to float64 and scaled by 2^-2log2(S) (exact).  (The
    paper's printed correction terms treat the matrix product elementwise;
    this is the exact expansion of Theorem 1's identity.)"""
    mS = qp.mS
    Si = 1 << qp.log2_scale
    out = np.empty(len(D))
    for i, d in enumerate(D):
        X = int(d) + mS * Si + 2 * mS * int(brow[i]) + mS * int(asum) + 2 * mS * mS * Nk
        out[i] = float(X) * (2.0 ** (-2 * qp.log2_scale))
    return out


# ------------------------------------------------------------- private ADMM


@dataclass
class PrivateTrace:
    x: list = field(default_factory=list)       # per round, float64 arrays
    z: list = field(default_factory=list)
    v: list = field(default_factory=list)
    D: list = field(default_factory=list)       # per round, decrypted integers
    xhat: list = field(default_factory=list)    # per round, x-hat ciphertexts (private_admm only)
    zhat: list = field(default_factory=list)
    vhat: list = field(default_factory=list)


def exact_rowdot(b, a) -> list:
    """Exact integers sum_j b_ij a_j for every row i of a non-negative int64
    matrix b (entries < 2^31) and non-negative ints a_j (< 2^31).

    Small problems use Python integers term by term.  Large ones split
    a_j = a_hi 2^16 + a_lo and take two int64 matrix-vector products (numpy,
    no floating point): every term b_ij a_lo < 2^47 and b_ij a_hi < 2^46, so
    both sums stay below 2^63 for rows of up to 2^15 terms; the two exact sums
    are recombined as Python integers."""
    b = np.asarray(b, dtype=np.int64)
    n = b.shape[1] if b.ndim == 2 else 0
    if b.size <= 1 << 16:
        return [sum(int(b[i, j]) * int(a[j]) for j in range(n)) for i in range(b.shape[0])]
    if n > 1 << 15 or np.any(b < 0) or np.any(b >= 1 << 31) or any(x < 0 or x >= 1 << 31 for x in a):
        raise ValueError("exact_rowdot: operand outside the split's range")
    av = np.asarray(a, dtype=np.int64)
    lo = b @ (av & 0xFFFF)
    hi = b @ (av >> 16)
    return [(int(h) << 16) + int(l) for h, l in zip(hi, lo)]


def _quantized_setup(setup: DisSetup, qp: QParams):
    c = [gamma1(a, qp) for a in setup.alpha]
    b = [gamma2(Bb, qp) for Bb in setup.Bbar]
    brow = [[int(s) for s in bk.sum(axis=1, dtype=np.int64)] for bk in b]
    return c, b, brow


def quantized_admm(setup: DisSetup, lam, rho, iters, qp: QParams) -> PrivateTrace:
    """Algorithm 1 with the decrypted plaintext replaced by the integer of
    Eq. (ret54), c_i + sum_j b_ij a_j, computed exactly with Python ints."""
    c, b, brow = _quantized_setup(setup, qp)
    N = setup.offsets[-1]
    z = np.zeros(N)
    v = np.zeros(N)
    tr = PrivateTrace()
    for _ in range(iters):
        zq = gamma2(z, qp)
        vq = gamma2(-v, qp)
        x = np.empty(N)
        Dall = []
        for k, (a0, a1) in enumerate(zip(setup.offsets[:-1], setup.offsets[1:])):
            a = [int(zq[j]) + int(vq[j]) for j in range(a0, a1)]
            D = [int(c[k][i]) + s for i, s in enumerate(exact_rowdot(b[k], a))]
            x[a0:a1] = decode(D, brow[k], sum(a), a1 - a0, qp)
            Dall.extend(D)
        z_new = soft_threshold(v + x, lam / rho)
        v = v + x - z_new
        z = z_new
        tr.x.append(x.copy())
        tr.z.append(z.copy())
        tr.v.append(v.copy())
        tr.D.append(Dall)
    return tr


def private_admm(setup: DisSetup, lam, rho, iters, qp: QParams, key: P.Key, seed: int) -> PrivateTrace:
    """Algorithm 1 of the paper with real Paillier encryption:

    setup   alpha-hat_k = E(Gamma1(alpha_k)) (Eq. (sldot2)); b_k = Gamma2(Bbar_k)
    round t master: z-hat = E(Gamma2(z)), (-v)-hat = E(Gamma2(-v)) (Eq. (uyt12))
            edge k: x-hat_k = alpha-hat_k (+) b_k (x) (z-hat_k (+) (-v)-hat_k) (Eq. (itq2))
            master: D = decrypt(x-hat), x = decode(D), z = S(v + x), v = v + x - z

    r for element e of vector `kind` in round t is r_of(key, seed,
    stream_id(t, kind), e) with e the global index."""
    c, b, brow = _quantized_setup(setup, qp)
    N = setup.offsets[-1]
    alpha_hat = P.encrypt(key, [int(v) for k in range(len(c)) for v in c[k]],
                          [P.r_of(key, seed, stream_id(0, KIND_ALPHA), e) for e in range(N)])
    z = np.zeros(N)
    v = np.zeros(N)
    tr = PrivateTrace()
    for t in range(1, iters + 1):
        zq = gamma2(z, qp)
        vq = gamma2(-v, qp)
        zhat = P.encrypt(key, [int(x) for x in zq], [P.r_of(key, seed, stream_id(t, KIND_Z), e) for e in range(N)])
        vhat = P.encrypt(key, [int(x) for x in vq], [P.r_of(key, seed, stream_id(t, KIND_V), e) for e in range(N)])
        x = np.empty(N)
        xhat_all, Dall = [], []
        for k, (a0, a1) in enumerate(zip(setup.offsets[:-1], setup.offsets[1:])):
            s = P.hom_add(key, zhat[a0:a1], vhat[a0:a1])
            xhat = P.hom_matvec(key, alpha_hat[a0:a1], s, b[k].astype(np.uint64))
            D = P.decrypt(key, xhat)
            a = [int(zq[j]) + int(vq[j]) for j in range(a0, a1)]
            x[a0:a1] = decode(D, brow[k], sum(a), a1 - a0, qp)
            xhat_all.extend(xhat)
            Dall.extend(D)
        z_new = soft_threshold(v + x, lam / rho)
        v = v + x - z_new
        z = z_new
        tr.x.append(x.copy())
        tr.z.append(z.copy())
        tr.v.append(v.copy())
        tr.D.append(Dall)
        tr.xhat.append(xhat_all)
        tr.zhat.append(zhat)
        tr.vhat.append(vhat)
    return tr


# ------------------------------------------------------------------ quantization error bound


def round_error_bound(setup: DisSetup, qp: QParams, z_prev, v_prev, x_priv) -> np.ndarray:
    """Per-element bound on |x_priv - x_plain| after one round from the same
    (z, v): the quantization errors of Eq. (et21) (half a step of Gamma1 on
    alpha, of Gamma2 on Bbar and on w = z - v) carried through the local
    update of Eq. (sldo091), plus one rounding of x:
    1/(2 S^2) + sum_j (|w~_j| / (2S) + |Bbar_ij| / S) + ulp(x_i)."""
    S = qp.S
    zq, vq = gamma2(z_prev, qp), gamma2(-np.asarray(v_prev), qp)
    wt = (zq + vq) / S + 2 * qp.zmin
    eps = np.empty(len(x_priv))
    for k, (a0, a1) in enumerate(zip(setup.offsets[:-1], setup.offsets[1:])):
        wsum = np.sum(np.abs(wt[a0:a1])) / (2 * S)
        rows = np.sum(np.abs(setup.Bbar[k]), axis=1) / S
        eps[a0:a1] = 0.5 / S ** 2 + wsum + rows + np.spacing(np.abs(x_priv[a0:a1]))
    return eps


def mse_gap_bound(setup: DisSetup, qp: QParams, xs, zs, vs, x_plain, x0) -> tuple[float, float]:
    """(Delta_T, bound on |MSE_priv - MSE_plain|) after T = len(xs) rounds of
    the private loop (iterates xs, zs, vs per round) against plaintext
    Dis-ADMM ending at x_plain.

    Scaled ADMM is Douglas-Rachford splitting on psi = z + v: with prox_f(u) =
    alpha + Bbar u (Eq. (sldo091); Bbar symmetric with eigenvalues in (0, 1],
    the proximal map of f(x) = sum_k ||y - A_k x_k||^2 / 2) and prox_g the soft
    threshold of Eq. (ty32), x^t = prox_f(2 prox_g(psi^{t-1}) - psi^{t-1}) and
    psi^t = T(psi^{t-1}) = x^t + v^{t-1}, with T firmly nonexpansive (the
    approximate-ADMM convergence argument the paper cites).  The private round
    computes x^t plus an error e_t bounded elementwise by round_error_bound,
    so ||psi_priv^t - psi^t|| <= sum_{s<=t} ||e_s|| and ||x_priv^T - x^T|| <=
    Delta_T = sum_{t<=T} ||eps_t||.  eps_t adds to the quantization terms the
    floating-point roundings of both runs: three ulps of |v| + |x| per run in
    the z/v updates, and the plaintext matvec's dot-product error
    gamma_{N_k+1} (|alpha_i| + sum_j |Bbar_ij| |w_j|) with |w_j| <= |w~_j| +
    Delta_{t-1}.  Then |MSE_priv - MSE_plain| <= (2 ||x_plain - x0|| Delta_T +
    Delta_T^2) / N."""
    N = len(x0)
    u = 2.0 ** -53
    dT = 0.0
    zp, vp = np.zeros(N), np.zeros(N)
    for t in range(len(xs)):
        eps = round_error_bound(setup, qp, zp, vp, xs[t])
        wt = np.abs((gamma2(zp, qp) + gamma2(-np.asarray(vp), qp)) / qp.S + 2 * qp.zmin) + dT
        for k, (a0, a1) in enumerate(zip(setup.offsets[:-1], setup.offsets[1:])):
            n = a1 - a0 + 1
            gam = n * u / (1 - n * u)
            eps[a0:a1] += gam * (np.abs(setup.alpha[k]) + np.abs(setup.Bbar[k]) @ wt[a0:a1])
        eps += 6 * np.spacing(np.abs(vp) + np.abs(xs[t]))
        dT += float(np.linalg.norm(eps))
        zp, vp = zs[t], vs[t]
    return dT, (2 * float(np.linalg.norm(np.asarray(x_plain) - x0)) * dT + dT ** 2) / N
