"""Seeded synthetic inputs for the tests, the benchmark and the smoke check.

This module only draws data: primes for keys, plaintexts, and the LASSO
problems of the paper's experiments (Sec. V: Gaussian A, sparse x0, noisy
y = A x0 + w).  It holds none of the method's arithmetic (no Paillier, no
quantizer, no ADMM), so both the CUDA library's callers and the CPU oracle can
consume the same inputs without sharing any computation.

Workloads (all seeded, all synthetic):

* ``lasso_small``   -- x0 in R^256 with 16 N(0,1) nonzeros at random
  positions; A 128x256 with N(0, 1/128) entries; y = A x0 + N(0, 0.01^2);
  split over 4 edge nodes; lambda 0.01, rho 1, 5 iterations; 1024-bit n.
* ``paillier_microbench`` -- 2^20 plaintexts rint(x * 2^24) + 2^47 with
  x ~ N(0,1) (about 48-bit integers), 2048-bit n, 16 groups of 2^16.
* ``lasso_large``   -- 256x256 image-like signal (N = 65536) with 5% nonzero
  DCT-domain coefficients, A (N/4) x N with N(0, 4/N) entries, 16 nodes,
  3072-bit n, 50 iterations, lambda 0.005, rho 1.
* ``batch_problem`` -- the batching form: 64 edge nodes with sizes
  log-uniform in [256, 65536], keys of 1024/2048/3072 bits assigned to the
  nodes in turn, an orthonormal design (A^T A = I), so only A^T y is drawn:
  x0 with 5% N(0,1) nonzeros plus N(0, 0.01^2) noise.
"""
from __future__ import annotations

import functools
import random
from dataclasses import dataclass

import numpy as np


@functools.lru_cache(maxsize=64)
def primes(nbits: int, seed: int) -> tuple[int, int]:
    """Two distinct primes of nbits/2 bits each, top two bits set, p < q.

    Drawn by seeding Python's Mersenne Twister and taking the next prime above
    a random odd start (sympy.nextprime, a library routine)."""
    import sympy

    half = nbits // 2
    rng = random.Random(seed * 1_000_003 + nbits)
    out = []
    while len(out) < 2:
        x = rng.getrandbits(half) | (3 << (half - 2)) | 1
        p = int(sympy.nextprime(x))
        if p.bit_length() == half and p not in out:
            out.append(p)
    p, q = sorted(out)
    return p, q


def plaintexts_u64(count: int, seed: int, scale_log2: int = 24, offset_log2: int = 47) -> np.ndarray:
    """Quantized-looking plaintexts: rint(x * 2^scale) + 2^offset with
    x ~ N(0, 1) (about offset+1 bits wide), as uint64."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(count)
    v = np.rint(x * float(2 ** scale_log2)).astype(np.int64) + (1 << offset_log2)
    return v.astype(np.uint64)


def uniform_below(bound: int, count: int, seed: int) -> list[int]:
    """count integers uniform in [0, bound) (Python Mersenne Twister)."""
    rng = random.Random(seed)
    return [rng.randrange(bound) for _ in range(count)]


@dataclass
class Lasso:
    A: np.ndarray      # M x N, float64
    y: np.ndarray      # M
    x0: np.ndarray     # N
    K: int             # edge nodes (column blocks)
    lam: float
    rho: float
    iters: int


def node_sizes(N: int, K: int) -> list[int]:
    """Column-block sizes for K edge nodes: as equal as possible."""
    base, extra = divmod(N, K)
    return [base + (1 if k < extra else 0) for k in range(K)]


def lasso_small(seed: int = 1, M: int = 128, N: int = 256, nnz: int = 16, K: int = 4, lam: float = 0.01,
                rho: float = 1.0, iters: int = 5, noise: float = 0.01) -> Lasso:
    """Sparse recovery problem of the paper's Sec. V (real Gaussian A)."""
    rng = np.random.default_rng(seed)
    x0 = np.zeros(N)
    pos = rng.choice(N, size=nnz, replace=False)
    x0[pos] = rng.standard_normal(nnz)
    A = rng.standard_normal((M, N)) / np.sqrt(M)
    y = A @ x0 + noise * rng.standard_normal(M)
    return Lasso(A=A, y=y, x0=x0, K=K, lam=lam, rho=rho, iters=iters)


def lasso_large(seed: int = 3, side: int = 256, frac: float = 0.05, K: int = 16, lam: float = 0.005, rho: float = 1.0,
                iters: int = 50, noise: float = 0.01, rows: int | None = None) -> Lasso:
    """Image-like signal: 5% of the side x side DCT coefficients nonzero, at
    positions drawn with probability proportional to 1/(1+u+v) (low
    frequencies favoured), values N(0,1); A has N(0, 4/N) entries and N/4
    rows (``rows`` overrides, for reduced checks)."""
    rng = np.random.default_rng(seed)
    N = side * side
    u, v = np.meshgrid(np.arange(side), np.arange(side), indexing="ij")
    w = (1.0 / (1.0 + u + v)).ravel()
    nnz = int(round(frac * N))
    pos = rng.choice(N, size=nnz, replace=False, p=w / w.sum())
    x0 = np.zeros(N)
    x0[pos] = rng.standard_normal(nnz)
    M = rows if rows is not None else N // 4
    A = rng.standard_normal((M, N)) * np.sqrt(4.0 / N)
    y = A @ x0 + noise * rng.standard_normal(M)
    return Lasso(A=A, y=y, x0=x0, K=K, lam=lam, rho=rho, iters=iters)


@dataclass
class BatchProblem:
    sizes: list          # N_k
    node_key: list       # index into key_bits per node
    key_bits: tuple
    x0: np.ndarray
    aty: np.ndarray      # A^T y, node by node (A^T A = I)
    lam: float
    rho: float


def batch_problem(seed: int = 5, nodes: int = 64, lo: int = 256, hi: int = 65536,
                  key_bits: tuple = (1024, 2048, 3072), frac: float = 0.05, noise: float = 0.01,
                  lam: float = 0.01, rho: float = 1.0) -> BatchProblem:
    """Edge-node sizes log-uniform in [lo, hi]; node k holds key key_bits[k % len].
    With orthonormal columns, A^T y = x0 + A^T w and A^T w ~ N(0, noise^2 I)."""
    rng = np.random.default_rng(seed)
    sizes = [int(round(float(np.exp(rng.uniform(np.log(lo), np.log(hi)))))) for _ in range(nodes)]
    N = sum(sizes)
    x0 = np.zeros(N)
    nnz = max(1, int(round(frac * N)))
    pos = rng.choice(N, size=nnz, replace=False)
    x0[pos] = rng.standard_normal(nnz)
    aty = x0 + noise * rng.standard_normal(N)
    return BatchProblem(sizes=sizes, node_key=[k % len(key_bits) for k in range(nodes)], key_bits=tuple(key_bits),
                        x0=x0, aty=aty, lam=lam, rho=rho)


def lasso_large_data(seed: int = 3, side: int = 256, frac: float = 0.05, K: int = 16, noise: float = 0.01,
                     device="cuda"):
    """The full-scale problem drawn node by node on a torch device (the dense
    A of N/4 x N doubles is 8.6 GB at N = 65536): x0 as lasso_large (numpy,
    5% nonzero DCT-domain coefficients, low frequencies favoured), A_k with
    N(0, 4/N) entries from a seeded torch generator, y = sum_k A_k x0_k +
    N(0, noise^2).  Returns (x0, node sizes, [A_k], y)."""
    import torch

    rng = np.random.default_rng(seed)
    N = side * side
    u, v = np.meshgrid(np.arange(side), np.arange(side), indexing="ij")
    w = (1.0 / (1.0 + u + v)).ravel()
    nnz = int(round(frac * N))
    pos = rng.choice(N, size=nnz, replace=False, p=w / w.sum())
    x0 = np.zeros(N)
    x0[pos] = rng.standard_normal(nnz)
    sizes = node_sizes(N, K)
    M = N // 4
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    xd = torch.from_numpy(x0).to(device)
    A, y, o = [], torch.zeros(M, dtype=torch.float64, device=device), 0
    for nk in sizes:
        Ak = torch.randn(M, nk, generator=g, dtype=torch.float64, device=device) * float(np.sqrt(4.0 / N))
        y += Ak @ xd[o:o + nk]
        A.append(Ak)
        o += nk
    y += noise * torch.randn(M, generator=g, dtype=torch.float64, device=device)
    return x0, sizes, A, y
