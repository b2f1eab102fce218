"""Benchmark of the Paillier hot path of 3P-ADMM-PC2 on B300.

Workload (one step): 2048-bit n, 2^20 quantized plaintexts rint(x 2^24) + 2^47
(x ~ N(0,1)); encrypt all of them (key-owner CRT path), aggregate the 16 node
groups of 2^16 by ciphertext products mod n^2, CRT-decrypt the 2^16
aggregates.  Metric: Paillier encryptions + decryptions per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs under torchrun, one rank per GPU, each rank on its own 2^20
plaintexts (weak scaling, no data-path collective).  --impl reference times
the CPU oracle (oracle/) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NBITS = 2048
N_PLAIN = 1 << 20
GROUPS = 16
SEED, STREAM = 0xB300, 1
METRIC = "Paillier enc/dec per s @2048-bit"
UNIT = "Paillier enc+dec ops/s"
# DRAM bytes (read + write) per element of k_enc_crt<64,1> from one ncu capture
# of this build (2^17 elements: 10.72 GB + 3.97 GB), scaled to a launch by the
# elements it processes; None once the kernel changes.
ENC_DRAM_BYTES_PER_ELEM = 112059
# DRAM bytes (read + write) per element of one k_modexp_tc launch from an ncu
# capture of this build (the power mod p^2 of 2^16 encryptions: 1.587 GB +
# 0.568 GB), scaled to a launch by the elements it processes; None once the
# kernel changes.
TC_DRAM_BYTES_PER_ELEM = 32886
WORKLOAD = "paillier_microbench: n=2048-bit, 2^20 plaintexts rint(N(0,1)*2^24)+2^47, encrypt (CRT) -> 16-group ciphertext product -> CRT decrypt of 2^16"
IMAD_PER_CLK_SM = 64   # nominal 32-bit integer multiply-add lanes per SM per clock (4 SMSPs x 16)
CPU_PER_GROUP = 4      # CPU sample: 16 x 4 encryptions, 16-group products, 4 decryptions per step


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def _oracle_sample(args):
    """One bounded oracle step: encrypt `per_group` plaintexts in each of 16
    groups, aggregate, decrypt the aggregates.  Runs in a worker process."""
    p, q, m_list, e_list, seed, stream = args
    from oracle import paillier as O

    ko = O.derive_key(p, q)
    c = O.encrypt(ko, m_list, [O.r_of(ko, seed, stream, e) for e in e_list])
    return c


def _cpu_reference(steps: int, warmup: int, per_group: int = CPU_PER_GROUP, workers: int | None = None):
    """Time the oracle (as it stands) on the host cores: each step encrypts
    16 x per_group plaintexts, multiplies the 16 groups, decrypts per_group
    aggregates, in a process pool of `workers` (default: every core).
    Returns (ops/s, cores, sample description, seconds/step)."""
    import concurrent.futures as cf
    import multiprocessing as mp

    from oracle import paillier as O
    from paper_2601_14980_b300 import workloads as W

    p, q = W.primes(NBITS, 2026)
    ko = O.derive_key(p, q)
    m = W.plaintexts_u64(GROUPS * per_group, seed=7)
    cores = workers or os.cpu_count() or 1
    work = [(p, q, [int(m[g * per_group + i])], [g * (N_PLAIN // GROUPS) + i], SEED, STREAM)
            for g in range(GROUPS) for i in range(per_group)]
    times = []
    with cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as ex:
        list(ex.map(_oracle_sample, work[:cores]))  # start the workers
        for s in range(warmup + steps):
            t0 = time.perf_counter()
            cts = [r[0] for r in ex.map(_oracle_sample, work)]
            groups = [cts[g * per_group:(g + 1) * per_group] for g in range(GROUPS)]
            agg = O.hom_sum(ko, groups)
            dec = list(ex.map(_dec_worker, [(p, q, a) for a in agg]))
            t1 = time.perf_counter()
            if s >= warmup:
                times.append(t1 - t0)
    per = statistics.mean(times)
    ops = GROUPS * per_group + per_group
    sample = ("%d encryptions + %d-group products + %d decryptions per step (of the 2^20 workload), mean of %d "
              "steps, process pool of %d" % (GROUPS * per_group, GROUPS, per_group, steps, cores))
    return ops / per, cores, sample, per


def _python_pow_reference(count: int = 8):
    """Secondary CPU reference, one thread: Eq. (itq1) and Sec. III-C with
    CPython's built-in three-argument pow on the same key and draws."""
    from oracle import paillier as O
    from paper_2601_14980_b300 import workloads as W

    p, q = W.primes(NBITS, 2026)
    ko = O.derive_key(p, q)
    m = [int(x) for x in W.plaintexts_u64(count, seed=7)]
    r = [O.r_of(ko, SEED, STREAM, e) for e in range(count)]
    t0 = time.perf_counter()
    c = [(1 + mi * ko.n) * pow(ri, ko.n, ko.n2) % ko.n2 for mi, ri in zip(m, r)]
    t1 = time.perf_counter()
    d = [(pow(ci, ko.lam, ko.n2) - 1) // ko.n * ko.mu % ko.n for ci in c]
    t2 = time.perf_counter()
    assert d == m
    return {"enc_per_s": count / (t1 - t0), "dec_per_s": count / (t2 - t1), "threads": 1,
            "sample": "%d encryptions and decryptions at 2048-bit n, CPython pow" % count}


def _dec_worker(args):
    p, q, c = args
    from oracle import paillier as O

    return O.decrypt(O.derive_key(p, q), [c])[0]


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _admm_setup(L, sizes):
    """Edge-node initialisation of Sec. II (input preparation, not timed):
    B_k = (A_k^T A_k + rho I)^-1, alpha_k = B_k A_k^T y, Bbar_k = rho B_k."""
    import numpy as np

    off = np.concatenate([[0], np.cumsum(sizes)]).astype(int)
    alpha, Bbar = [], []
    for k in range(len(sizes)):
        Ak = L.A[:, off[k]:off[k + 1]]
        Bk = np.linalg.inv(Ak.T @ Ak + L.rho * np.eye(sizes[k]))
        alpha.append(Bk @ (Ak.T @ L.y))
        Bbar.append((L.rho * Bk).ravel())
    return np.concatenate(alpha), np.concatenate(Bbar)


def _mse_gap_bound(ctx, sizes, alpha, Bbar, xs, zs, vs, x_plain, x0, zmin: float, log2_scale: int):
    """Bound on |MSE_priv - MSE_plain| after len(xs) private rounds.  Scaled
    ADMM is Douglas-Rachford on psi = z + v with a firmly nonexpansive
    operator, so the per-round errors of x add up at most linearly:
    Delta_T = sum_t ||eps_t|| with, per element, the quantization errors
    carried through the local update, 1/(2 S^2) + sum_j (|w~_j| / (2S) +
    |Bbar_ij| / S), one rounding of x, three ulps of |v| + |x| per run in the
    z/v updates, and the plaintext matvec's dot-product error; then the MSE
    gap is at most (2 ||x_plain - x0|| Delta_T + Delta_T^2) / N.  Tensors on
    the device."""
    import torch

    from paper_2601_14980_b300 import pc2

    S = float(2 ** log2_scale)
    u = 2.0 ** -53
    N = int(sum(sizes))
    off = [0]
    for n in sizes:
        off.append(off[-1] + int(n))
    blocks, b0 = [], 0
    for n in sizes:
        blocks.append(Bbar[b0:b0 + n * n].view(n, n).abs())
        b0 += n * n
    rowabs = torch.cat([b.sum(dim=1) for b in blocks]) / S
    inf = torch.tensor(float("inf"), dtype=torch.float64, device=Bbar.device)

    def ulp(a):
        a = a.abs()
        return torch.nextafter(a, inf) - a

    dT = 0.0
    zp = torch.zeros(N, dtype=torch.float64, device=Bbar.device)
    vp = torch.zeros_like(zp)
    for t in range(len(xs)):
        zq = pc2.quantize(ctx, zp, zmin, -zmin, log2_scale, 2).double()
        vq = pc2.quantize(ctx, vp, zmin, -zmin, log2_scale, 2, negate=True).double()
        wt = ((zq + vq) / S + 2 * zmin).abs()
        eps = torch.empty(N, dtype=torch.float64, device=Bbar.device)
        for k in range(len(sizes)):
            a0, a1 = off[k], off[k + 1]
            n = a1 - a0 + 1
            gam = n * u / (1 - n * u)
            eps[a0:a1] = wt[a0:a1].sum() / (2 * S) + gam * (alpha[a0:a1].abs() + blocks[k] @ (wt[a0:a1] + dT))
        x = xs[t]
        eps += 0.5 / S ** 2 + rowabs + ulp(x) + 6 * ulp(vp.abs() + x.abs())
        dT += float(torch.linalg.norm(eps))
        zp, vp = zs[t], vs[t]
    gap = (2 * float(torch.linalg.norm(x_plain - x0)) * dT + dT ** 2) / N
    return dT, gap


def run_admm(dev, rounds: int = 5):
    """Seconds per ADMM iteration on the small LASSO workload (1024-bit n,
    4 nodes): batched rounds (one graph per round) vs the per-node path."""
    import numpy as np
    import torch

    from paper_2601_14980_b300 import pc2
    from paper_2601_14980_b300 import workloads as W

    L = W.lasso_small(seed=1)
    sizes = W.node_sizes(L.A.shape[1], L.K)
    alpha, Bbar = _admm_setup(L, sizes)
    da, dB = torch.from_numpy(alpha).to(dev), torch.from_numpy(Bbar).to(dev)
    ctx = pc2.Context(dev)
    key = pc2.Key.generate(1024, 2026)
    out = {}
    st = torch.cuda.current_stream()
    for name, per_node in (("batched", False), ("per_node", True)):
        adm = pc2.Admm(ctx, key, sizes, da, dB, L.lam, L.rho, -8.0, 8.0, 24, 77, per_node=per_node)
        adm.round(2)                      # warm-up (first round eager, graph captured)
        adm.reset()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        adm.round(rounds)
        b.record(st)
        b.synchronize()
        out[name] = a.elapsed_time(b) / 1e3 / rounds
        if name == "batched":
            # the same rounds again, one at a time, keeping the iterates for the bound
            adm.reset()
            xs, zs, vs = [], [], []
            for _ in range(rounds):
                adm.round(1)
                x, z, v, _ = adm.get()
                xs.append(x.clone()), zs.append(z.clone()), vs.append(v.clone())
            out["mse"] = float(np.mean((xs[-1].cpu().numpy() - L.x0) ** 2))
            adm.reset()
            torch.cuda.synchronize()
            a.record(st)
            adm.round_plain(rounds)
            b.record(st)
            b.synchronize()
            out["plain_dis_admm"] = a.elapsed_time(b) / 1e3 / rounds
            xp = adm.get()[0].clone()
            out["mse_plain"] = float(np.mean((xp.cpu().numpy() - L.x0) ** 2))
            x0 = torch.from_numpy(L.x0).to(dev)
            out["delta_T"], out["bound"] = _mse_gap_bound(ctx, sizes, da, dB, xs, zs, vs, xp, x0, -8.0, 24)
        adm.close()
    return {"workload": "lasso_small: A 128x256, 4 edge nodes, 1024-bit n, %d rounds" % rounds,
            "s_per_iter_batched": out["batched"], "s_per_iter_per_node": out["per_node"],
            "batched_speedup": out["per_node"] / out["batched"], "s_per_iter_plaintext_dis_admm": out["plain_dis_admm"],
            "mse_private": out["mse"], "mse_plaintext": out["mse_plain"],
            "mse_gap": abs(out["mse"] - out["mse_plain"]), "mse_bound": out["bound"], "delta_T": out["delta_T"],
            "within_bound": abs(out["mse"] - out["mse_plain"]) <= out["bound"]}


def run_admm_full(dev, rounds: int = 2):
    """Full-scale private ADMM: 256 x 256 image-like LASSO (N = 65536, 16 edge
    nodes of 4096, A of N/4 x N), 3072-bit n, lambda 0.005, rho 1.  Seconds per
    round of the batched path (round 1 eager, then the captured graph) and of
    the per-node path."""
    import numpy as np
    import torch

    from paper_2601_14980_b300 import pc2
    from paper_2601_14980_b300 import workloads as W

    x0, sizes, A, y = W.lasso_large_data(device=dev)
    rho, lam = 1.0, 0.005
    alphas, bbars = [], []
    for Ak in A:
        B = torch.linalg.inv(Ak.T @ Ak + rho * torch.eye(Ak.shape[1], dtype=torch.float64, device=Ak.device))
        alphas.append(B @ (Ak.T @ y))
        bbars.append((rho * B).reshape(-1))
    del A
    alpha, Bbar = torch.cat(alphas), torch.cat(bbars)
    del alphas, bbars
    ctx = pc2.Context(dev)
    key = pc2.Key.generate(3072, 2028)
    st = torch.cuda.current_stream()
    out = {}
    for name, per_node in (("batched", False), ("per_node", True)):
        adm = pc2.Admm(ctx, key, sizes, alpha, Bbar, lam, rho, -8.0, 8.0, 24, 77, per_node=per_node)
        ms = 0.0
        xs, zs, vs = [], [], []
        for _ in range(rounds):          # round 1 eager, then the captured graph
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            adm.round(1)
            b.record(st)
            b.synchronize()
            ms += a.elapsed_time(b)
            if name == "batched":
                x, z, v, _ = adm.get()
                xs.append(x.clone()), zs.append(z.clone()), vs.append(v.clone())
        out[name] = ms / 1e3 / rounds
        if name == "batched":
            x0d = torch.from_numpy(x0).to(dev)
            out["mse"] = float(((xs[-1] - x0d) ** 2).mean())
            out["matvec"] = adm.info()
            adm.reset()
            adm.round_plain(rounds)
            xp = adm.get()[0].clone()
            out["mse_plain"] = float(((xp - x0d) ** 2).mean())
            out["delta_T"], out["bound"] = _mse_gap_bound(ctx, sizes, alpha, Bbar, xs, zs, vs, xp, x0d, -8.0, 24)
            del xs, zs, vs
        adm.close()
    return {"workload": "lasso_large: N=65536 (256x256, 5%% DCT nonzeros), 16 edge nodes, A %dx%d, 3072-bit n, "
                        "%d rounds" % (len(y), len(x0), rounds),
            "s_per_iter_batched": out["batched"], "s_per_iter_per_node": out["per_node"],
            "batched_speedup": out["per_node"] / out["batched"], "mse_after_rounds": out["mse"],
            "mse_plaintext_after_rounds": out["mse_plain"], "mse_gap": abs(out["mse"] - out["mse_plain"]),
            "mse_bound": out["bound"], "delta_T": out["delta_T"],
            "within_bound": abs(out["mse"] - out["mse_plain"]) <= out["bound"],
            "matvec": out["matvec"], "status": ctx.status()}


def run_batch(dev, rounds: int = 1, per_node_rounds: int = 1, tune: bool = True):
    """Batching form: 64 edge nodes, sizes log-uniform in [256, 65536], keys of
    1024/2048/3072 bits (one per size, nodes assigned in turn), orthonormal
    design (Bbar diagonal).  Seconds per round of the persistent batched launch
    (CUDA graph) vs the plain per-node path on the same GPU, and the MSE of x
    after the batched rounds."""
    import numpy as np
    import torch

    from paper_2601_14980_b300 import pc2
    from paper_2601_14980_b300 import workloads as W

    bp = W.batch_problem()
    rho = bp.rho
    # Sec. II initialization for A^T A = I: alpha = A^T y / (1 + rho), Bbar = rho / (1 + rho) I
    alpha = torch.from_numpy(bp.aty / (1.0 + rho)).to(dev)
    bdiag = torch.full((len(bp.aty),), rho / (1.0 + rho), dtype=torch.float64, device=dev)
    ctx = pc2.Context(dev)
    keys = [pc2.Key.generate(b, 2026 + b) for b in bp.key_bits]
    st = torch.cuda.current_stream()
    t0 = time.time()
    bt = pc2.Batch(ctx, keys, bp.sizes, bp.node_key, alpha, bdiag, bp.lam, rho, -8.0, 8.0, 24, 77)
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    tuned = bt.tune() if tune else None
    info = bt.info()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = Clocks(dev)
    a.record(st)
    bt.round(rounds)
    b.record(st)
    b.synchronize()
    batched = a.elapsed_time(b) / 1e3 / rounds
    clocks = clk.stop()
    x = bt.get()[0].cpu().numpy()
    mse = float(np.mean((x - bp.x0) ** 2))
    bt.reset()
    a.record(st)
    bt.round_per_node(per_node_rounds)
    b.record(st)
    b.synchronize()
    per_node = a.elapsed_time(b) / 1e3 / per_node_rounds
    status = ctx.status()
    bt.close()
    N = info["elements"]
    return {"workload": "batch_problem: 64 edge nodes, sizes log-uniform [256, 65536] (N=%d), keys 1024/2048/3072-bit "
                        "(one per size, nodes in turn), orthonormal design" % N,
            "elements": N, "work_items": info["items"], "grid": info["grid"],
            "scratch_gb": info["scratch_bytes"] / 1e9, "tuned": tuned, "setup_s": setup_s,
            "s_per_round_batched": batched, "s_per_round_per_node": per_node,
            "batched_speedup": per_node / batched, "elements_per_s_batched": N / batched,
            "rounds_batched": rounds, "rounds_per_node": per_node_rounds, "mse_after_batched_rounds": mse,
            "status": status, "clocks": clocks}


def run_serve(dev, rates=(5.0, 15.0, 30.0, 45.0, 60.0), seconds: float = 4.0, seed: int = 11):
    """Serving form: Poisson arrivals of encrypt / decrypt / aggregate requests
    (one third each) from 256 simulated edge nodes, 2048-bit n, sizes
    log-uniform in [64, 32768] ciphertexts, aggregates of 2..16 node vectors,
    payloads rint(N(0,1) 2^24) + 2^47; device-resident key and request buffers
    with memory admission.  p50/p99 latency and ciphertexts/s per arrival rate
    for continuous batching (mode 0) and the plain per-request path (mode 1)."""
    import numpy as np
    import torch

    from paper_2601_14980_b300 import pc2
    from paper_2601_14980_b300 import workloads as W

    ctx = pc2.Context(dev)
    key = pc2.Key.generate(2048, 2027)
    L, L2 = key.limbs, 2 * key.limbs
    MAXC, GMAX = 32768, 16
    m = W.plaintexts_u64(MAXC, seed=seed)
    h_m = torch.from_numpy(m.view(np.int64)).pin_memory()
    dm = h_m.to(dev)
    stride = pc2.tiled_words(MAXC, L2)
    pool = torch.empty(GMAX * stride, dtype=torch.int32, device=dev)
    for g in range(GMAX):
        pc2.encrypt(ctx, key, dm, seed, 1000 + g, 0, out=pool[g * stride:(g + 1) * stride])
    h_pool = pool.cpu().pin_memory()
    del pool
    rng = np.random.default_rng(seed)
    points = []
    for rate in rates:
        n = max(20, int(rate * seconds))
        arr = np.cumsum(rng.exponential(1.0 / rate, n))
        ops = rng.integers(1, 4, n)
        counts = np.exp(rng.uniform(np.log(64), np.log(MAXC), n)).astype(int)
        groups = rng.integers(2, GMAX + 1, n)
        nodes = rng.integers(0, 256, n)
        outw = [pc2.tiled_words(int(c), L if o == pc2.OP_DECRYPT else L2) for o, c in zip(ops, counts)]
        offs = np.concatenate([[0], np.cumsum(outw)]).astype(int)
        h_out = torch.empty(int(offs[-1]), dtype=torch.int32).pin_memory()
        res = {"rate_per_s": rate, "requests": n, "ciphertexts": int(counts.sum())}
        for mode, name in ((0, "batched"), (1, "per_request")):
            srv = pc2.Server(ctx, key, arena_bytes=4 << 30, mode=mode)
            t0 = time.perf_counter()
            tickets, sub = [], []
            for i in range(n):
                d = t0 + arr[i] - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                o, c = int(ops[i]), int(counts[i])
                out = h_out[offs[i]:offs[i + 1]]
                if o == pc2.OP_ENCRYPT:
                    h_in = h_m
                elif o == pc2.OP_DECRYPT:
                    h_in = h_pool
                else:
                    h_in = h_pool
                sub.append(time.perf_counter())
                tickets.append(srv.submit(o, h_in, c, out, groups=int(groups[i]), seed=seed, stream=int(nodes[i]),
                                          e0=int(rng.integers(0, 1 << 20)), h_stride=stride))
            lats = [srv.wait(t) for t in tickets]
            span = max(s + l for s, l in zip(sub, lats)) - t0
            st = srv.stats()
            srv.close()
            worst = sorted(range(n), key=lambda i: -lats[i])[:3]
            res[name] = {"p50_s": float(np.percentile(lats, 50)), "p99_s": float(np.percentile(lats, 99)),
                         "ciphertexts_per_s": int(counts.sum()) / span, "makespan_s": span, "steps": st["steps"],
                         "slowest": [{"op": int(ops[i]), "count": int(counts[i]), "latency_s": lats[i]} for i in worst]}
        points.append(res)
    return {"workload": "serving: Poisson arrivals from 256 edge nodes, 2048-bit n, sizes log-uniform [64, 32768], "
                        "encrypt/decrypt/aggregate(2..16) in equal shares, %.0f s per rate" % seconds,
            "points": points, "status": ctx.status()}


# The paper's Table II, master node GPU (RTX 4060), for context only: ops/s.
PAPER_TABLE2_RTX4060 = {
    1024: {"modmult": 4062.66e3, "modexp": 79352.5, "ep": 137807.85},
    2048: {"modmult": 1544.13e3, "modexp": 31080.16, "ep": 65662.72},
    4096: {"modmult": 1414.34e3, "modexp": 26594.01, "ep": 50053.47},
}


def run_tc_mont(dev, count: int = 1 << 20, nsq: int = 64, reps: int = 3):
    """The tensor-core experiment: nsq Montgomery squarings of `count`
    elements mod N = p^2 (2048 bits) of the benchmark's key, with the
    reduction's contractions on tcgen05 (f16 digits) vs the integer-pipe
    CIOS product.  Inputs resident in device memory, CUDA events, mean of
    `reps` after one warm-up; both results compared word for word."""
    import torch

    from paper_2601_14980_b300 import pc2

    ctx = pc2.Context(dev)
    p = pc2.Key.generate(NBITS, 2026).export()["p"]
    N = p * p
    g = torch.Generator(device=dev).manual_seed(9)
    canon = torch.randint(-(1 << 31), 1 << 31, (count, 64), generator=g, dtype=torch.int64, device=dev)
    canon[:, 63] = torch.randint(0, (N >> 2016) - 1, (count,), generator=g, device=dev)   # x < N
    x = pc2.pack(ctx, canon.to(torch.int32).reshape(-1), count, 64)
    st = torch.cuda.current_stream()
    out, res = {}, {}
    for name, eng in (("imad_cios", pc2.ENGINE_IMAD), ("tensor_core", pc2.ENGINE_TC)):
        y = pc2.empty_tiled(count, 64)
        pc2.mont_sqr(ctx, N, x, count, nsq, eng, out=y)
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            pc2.mont_sqr(ctx, N, x, count, nsq, eng, out=y)
            b.record(st)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        t = statistics.mean(ms)
        prods = count * nsq * (2 * 64 * 64 + 64)
        out[name] = {"ms": t, "squarings_per_s": count * nsq / (t / 1e3), "t_word_products_per_s": prods / t / 1e9}
        res[name] = y
    same = bool(torch.equal(pc2.unpack(ctx, res["imad_cios"], count, 64), pc2.unpack(ctx, res["tensor_core"], count, 64)))
    return {"workload": "%d elements x %d Montgomery squarings mod p^2 (2048 bits)" % (count, nsq), "engines": out,
            "tc_over_imad": out["imad_cios"]["ms"] / out["tensor_core"]["ms"], "bit_identical": same,
            "status": ctx.status()}


def run_table2(dev, count: int = 9000, trials: int = 10):
    """Throughput of the operations of the paper's Table II on B300, on its
    workload: 9000 plaintexts uniform in [0, n), modulus n^2, mean of 10
    trials, at n = 1024, 2048 and 4096.  ModMult = one product of two
    ciphertexts mod n^2 (pc2_hom_add); ModExp = c^k mod n^2 with k uniform in
    [0, n) (pc2_hom_scal_wide); EP = the key-owner encryption of a plaintext
    in [0, n) through the CRT halves (pc2_encrypt_wide); also public-key
    encryption (64-bit plaintexts) and CRT decryption.  Inputs resident in
    device memory; each trial timed with CUDA events after one warm-up."""
    import torch

    from paper_2601_14980_b300 import pc2
    from paper_2601_14980_b300 import workloads as W

    ctx = pc2.Context(dev)
    st = torch.cuda.current_stream()
    rows = {}
    for nbits in (1024, 2048, 4096):
        key = pc2.Key.generate(nbits, 2026)
        n = key.export()["n"]
        L, L2 = key.limbs, 2 * key.limbs
        m = pc2.ints_to_tiled(ctx, W.uniform_below(n, count, nbits), L)
        kexp = pc2.ints_to_tiled(ctx, W.uniform_below(n, count, nbits + 1), L)
        m64 = torch.from_numpy(W.plaintexts_u64(count, seed=nbits).view("int64")).to(dev)
        ct = pc2.encrypt_wide(ctx, key, m, count, SEED, STREAM)
        ct2 = pc2.encrypt_wide(ctx, key, m, count, SEED, STREAM + 1)
        out = pc2.empty_tiled(count, L2)
        dec = pc2.empty_tiled(count, L)
        ops = {
            "modmult": lambda: pc2.hom_add(ctx, key, ct, ct2, count, out=out),
            "modexp": lambda: pc2.hom_scal_wide(ctx, key, ct, kexp, count, out=out),
            "ep": lambda: pc2.encrypt_wide(ctx, key, m, count, SEED, STREAM, out=out),
            "encrypt_public": lambda: pc2.encrypt(ctx, key, m64, SEED, STREAM, out=out, public=True),
            "decrypt": lambda: pc2.decrypt(ctx, key, ct, count, out=dec),
        }
        row = {}
        for name, fn in ops.items():
            fn()
            torch.cuda.synchronize()
            ms = []
            for _ in range(trials):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(st)
                fn()
                b.record(st)
                b.synchronize()
                ms.append(a.elapsed_time(b))
            row[name] = count / (statistics.mean(ms) / 1e3)
        assert ctx.status() == 0
        paper = PAPER_TABLE2_RTX4060[nbits]
        row["paper_rtx4060"] = paper
        row["ratio_to_paper"] = {k: row[k] / paper[k] for k in paper}
        rows[str(nbits)] = row
        del ct, ct2, out, dec, m, kexp
    return {"workload": "Table II: %d plaintexts uniform in [0, n), modulus n^2, mean of %d trials" % (count, trials),
            "unit": "ops/s", "rows": rows}


def run_hbm(dev, n: int = 1 << 27, n_dec: int = 1 << 24, reps: int = 5):
    """Achieved HBM bandwidth of the memory-bound steps on vectors far larger
    than L2 (each input 1 GiB at n = 2^27): quantize (Gamma2, Eq. (et21)),
    dequantize, the z/v update (Eqs. (ty32), (u78)) and the exact decode of
    Theorem 1 on 1024-bit decrypted rows.  GB/s = algorithmic bytes (inputs
    read once, outputs written once) / CUDA-event time, mean of `reps`."""
    import torch

    from paper_2601_14980_b300 import pc2

    ctx = pc2.Context(dev)
    st = torch.cuda.current_stream()
    g = torch.Generator(device=dev).manual_seed(5)
    u = torch.randn(n, generator=g, dtype=torch.float64, device=dev)
    q = torch.empty(n, dtype=torch.int64, device=dev)
    x = torch.randn(n, generator=g, dtype=torch.float64, device=dev) * 0.02
    z = torch.zeros(n, dtype=torch.float64, device=dev)
    v = torch.randn(n, generator=g, dtype=torch.float64, device=dev) * 0.02
    limbs = 32
    # decrypted rows below 2^62 (words 0, 1; the other words zero, as the decode expects),
    # tiled: words 0..3 of a tile's 32 elements form its first 128-word slab
    D = torch.zeros(pc2.tiled_words(n_dec, limbs), dtype=torch.int32, device=dev)
    lo = D.view(-1, limbs // 4, 32, 4)[:, 0]
    lo[:, :, 0] = torch.randint(-(1 << 31), 1 << 31, lo[:, :, 0].shape, generator=g, dtype=torch.int32, device=dev)
    lo[:, :, 1] = torch.randint(0, 1 << 30, lo[:, :, 1].shape, generator=g, dtype=torch.int32, device=dev)
    brow = torch.randint(0, 1 << 30, (n_dec,), generator=g, dtype=torch.int64, device=dev)
    asum = torch.randint(0, 1 << 33, (n_dec,), generator=g, dtype=torch.int64, device=dev)
    nk = torch.full((n_dec,), 64, dtype=torch.int32, device=dev)
    xd = torch.empty(n_dec, dtype=torch.float64, device=dev)
    steps = {
        "quantize": (lambda: pc2.quantize(ctx, u, -8.0, 8.0, 24, 2, out=q), 16 * n),
        "dequantize": (lambda: pc2.dequantize(ctx, q, -8.0, 24, 2, out=u), 16 * n),
        "zv_update": (lambda: pc2.zv_update(ctx, x, z, v, 0.01), 32 * n),   # x, v in; z, v out
        "decode_matvec": (lambda: pc2.decode_matvec(ctx, D, limbs, n_dec, brow, asum, nk, -8.0, 24, out=xd),
                          (4 * limbs + 8 + 8 + 4 + 8) * n_dec),
    }
    peak = _peaks().get("hbm_gbs")
    out = {}
    for name, (fn, nbytes) in steps.items():
        fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            fn()
            b.record(st)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        t = statistics.mean(ms)
        gbs = nbytes / (t / 1e3) / 1e9
        out[name] = {"elements": n if name != "decode_matvec" else n_dec, "bytes": nbytes, "ms": t, "gb_s": gbs,
                     "frac_of_measured_hbm": gbs / peak if peak else None}
    del u, q, x, z, v, D, brow, asum, nk, xd
    torch.cuda.empty_cache()
    return {"peak_gb_s": peak, "peak_note": "MEASURED_PEAKS.json hbm_gbs (copy, read + write)", "steps": out}


def run_probe(dev) -> dict:
    """Measured rates of the 32-bit multiplies on this GPU (pc2_probe_mul):
    mad.lo, mad.hi, mad.wide (a whole 32x32->64 product), a product as
    mad.lo + mad.hi, the carry-chained rows of a 64-limb Montgomery
    product (the integer-pipe engine) and the same rows as wide products
    with 64-bit adds (the tensor-core engine's integer half), both at 3 CTAs
    of 128 per SM, and the FP64 add rate.
    Per SM and clock from clock64 inside the loops; per second from CUDA
    events around each launch (after one untimed warm-up launch)."""
    from paper_2601_14980_b300 import pc2

    kinds = [("mad_lo", pc2.PROBE_LO, 8, 40000), ("mad_hi", pc2.PROBE_HI, 8, 20000),
             ("mad_wide", pc2.PROBE_WIDE, 8, 20000), ("lo_hi_product", pc2.PROBE_LOHI, 8, 15000),
             ("cios_row_64_limbs", pc2.PROBE_ROW, 3, 600), ("wide_row_64_limbs", pc2.PROBE_ROWW, 3, 600),
             ("fp64_add", pc2.PROBE_DADD, 8, 2000)]
    out = {}
    clk = Clocks(dev)
    for name, kind, bps, iters in kinds:
        pc2.probe_mul(dev, kind, bps, max(1, iters // 10))
        r = pc2.probe_mul(dev, kind, bps, iters)
        out[name] = {"per_clk_per_sm": r["ops"] / (r["cycles"] * r["sms"]), "per_s": r["ops"] / (r["ms"] / 1e3),
                     "ms": r["ms"], "ctas_per_sm": bps, "sm_mhz": r["cycles"] / (r["ms"] * 1e3)}
    out["clocks"] = clk.stop()
    wide, lohi = out["mad_wide"]["per_s"], out["lo_hi_product"]["per_s"]
    out["product_peak_per_s"] = max(wide, lohi)
    out["product_peak_kind"] = "mad_wide" if wide >= lohi else "lo_hi_product"
    return out


def run_gpu(args):
    import numpy as np
    import torch

    from paper_2601_14980_b300 import pc2
    from paper_2601_14980_b300 import workloads as W

    from paper_2601_14980_b300.dist import max_over_ranks, rank_world, shard

    rank, world, local = rank_world()
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    cpu_base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sample, per = _cpu_reference(steps=3, warmup=1)
        v1, _, sample1, _ = _cpu_reference(steps=1, warmup=0, per_group=1, workers=1)
        cpu_base = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                    "single_thread": {"value": v1, "sample": sample1},
                    "python_pow": _python_pow_reference()}

    global N_PLAIN, GROUPS
    N_PLAIN, GROUPS = args.plaintexts, args.groups
    ctx = pc2.Context(dev)
    pc2.set_engine(ctx, args.engine)
    key = pc2.Key.generate(NBITS, 2026)
    L2 = 2 * key.limbs
    per_group = N_PLAIN // GROUPS
    m_host = W.plaintexts_u64(N_PLAIN, seed=7 + rank)
    m_pinned = torch.from_numpy(m_host.view(np.int64)).pin_memory()
    dm = m_pinned.to(f"cuda:{dev}")
    ct = torch.empty(pc2.tiled_words(N_PLAIN, L2), dtype=torch.int32, device=dev)
    agg = torch.empty(pc2.tiled_words(per_group, L2), dtype=torch.int32, device=dev)
    dec = torch.empty(pc2.tiled_words(per_group, key.limbs), dtype=torch.int32, device=dev)
    dec_host = torch.empty(dec.numel(), dtype=torch.int32).pin_memory()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 126 MB L2
    st = torch.cuda.current_stream()
    e0, _ = shard(world * N_PLAIN, rank, world)   # this rank's elements are global indices e0 ..

    def step(ev=None, e2e=False):
        if e2e:
            dm.copy_(m_pinned, non_blocking=True)
        if ev: ev[0].record(st)
        pc2.encrypt(ctx, key, dm, SEED, STREAM, e0=e0, out=ct)
        if ev: ev[1].record(st)
        pc2.hom_sum(ctx, key, ct, GROUPS, per_group, out=agg)
        if ev: ev[2].record(st)
        pc2.decrypt(ctx, key, agg, per_group, out=dec)
        if ev: ev[3].record(st)
        if e2e:
            dec_host.copy_(dec, non_blocking=True)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ctx.status() != 0:
        raise RuntimeError("device status raised during warm-up")

    clocks = Clocks(dev) if rank == 0 else None
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    if dist: dist.barrier()
    torch.cuda.synchronize()
    for s in range(args.steps):
        flush.zero_()
        step(evs[s])
    torch.cuda.synchronize()
    if dist: dist.barrier()
    clk = clocks.stop() if clocks else None
    t_enc = [evs[s][0].elapsed_time(evs[s][1]) for s in range(args.steps)]
    t_sum = [evs[s][1].elapsed_time(evs[s][2]) for s in range(args.steps)]
    t_dec = [evs[s][2].elapsed_time(evs[s][3]) for s in range(args.steps)]
    step_ms = [a + b + c for a, b, c in zip(t_enc, t_sum, t_dec)]
    ms = statistics.mean(step_ms)

    # end to end: host plaintexts in, host plaintexts out, through the C ABI
    e2e_ms = []
    for s in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        step(None, e2e=True)
        b.record(st)
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    ms_e2e = statistics.mean(e2e_ms)

    ms, ms_e2e = max_over_ranks([ms, ms_e2e], device=dev)
    ops = (N_PLAIN + per_group) * world
    value = ops / (ms / 1e3)

    # the same encryption and decryption on each engine of the full-width
    # powers (integer pipe; tensor cores), outside the step
    engine_ab = None
    if rank == 0 and not args.no_engine_ab:
        engine_ab = {}
        for name, eng in (("imad", pc2.ENGINE_IMAD), ("tensor_core", pc2.ENGINE_TC)):
            pc2.set_engine(ctx, eng)
            r = {}
            for op, fn in (("encrypt_ms", lambda: pc2.encrypt(ctx, key, dm, SEED, STREAM, e0=e0, out=ct)),
                           ("decrypt_2p16_ms", lambda: pc2.decrypt(ctx, key, agg, per_group, out=dec))):
                fn()
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(st)
                fn()
                b.record(st)
                b.synchronize()
                r[op] = a.elapsed_time(b)
            engine_ab[name] = r
        pc2.set_engine(ctx, args.engine)
        assert ctx.status() == 0

    # stage times of the tensor-core path (CUDA events recorded by the library
    # on this stream around each of its launches), one encryption of the batch
    # and one decryption of the aggregates
    stages = None
    if rank == 0 and args.engine != 0:
        def timed_stages(fn):
            flush.zero_()
            fn()
            try:
                return dict(zip(["setup", "power_p2", "power_q2", "finish"], pc2.stage_ms(ctx)))
            except pc2.Pc2Error:    # the call ran on the integer-pipe engine (below its size threshold)
                return None
        pc2.set_timing(ctx, True)
        stages = {"encrypt": timed_stages(lambda: pc2.encrypt(ctx, key, dm, SEED, STREAM, e0=e0, out=ct)),
                  "decrypt_2p16": timed_stages(lambda: pc2.decrypt(ctx, key, agg, per_group, out=dec))}
        pc2.set_timing(ctx, False)

    # decryption of the whole batch (all 2^20 ciphertexts), outside the step
    dec_full_ms = None
    if rank == 0:
        dec_full = torch.empty(pc2.tiled_words(N_PLAIN, key.limbs), dtype=torch.int32, device=dev)
        reps = []
        for _ in range(2):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            pc2.decrypt(ctx, key, ct, N_PLAIN, out=dec_full)
            b.record(st)
            b.synchronize()
            reps.append(a.elapsed_time(b))
        dec_full_ms = statistics.mean(reps)
        del dec_full

    # roofline of the dominant kernel (encryption): algorithmic 32x32->64
    # word products / time, against the measured product rate of the multiplier
    mm, mmh, lb = key.cost(ctx, pc2.COST_ENCRYPT)
    imad_per_elem = key.imads(ctx, pc2.COST_ENCRYPT)
    prod_enc = key.products(ctx, pc2.COST_ENCRYPT)
    prod_dec = key.products(ctx, pc2.COST_DECRYPT)
    prod_sum = GROUPS * (2 * L2 * L2 + L2)      # (groups - 1) products and the R^k fix-up, n^2 limbs
    enc_ms = statistics.mean(t_enc)
    dec_ms = statistics.mean(t_dec)
    sum_ms = statistics.mean(t_sum)
    peaks = _peaks()
    sm_max = peaks.get("sm_max_mhz", 2032.0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    nominal_imad = sms * IMAD_PER_CLK_SM * sm_max * 1e6 / 1e12
    probe = None
    if rank == 0 and not args.no_probe:
        probe = run_probe(dev)
    dmm, _, dlb = key.cost(ctx, pc2.COST_DECRYPT)
    if rank != 0:
        if dist: dist.destroy_process_group()
        return
    ach_enc = prod_enc * N_PLAIN / (enc_ms / 1e3) / 1e12
    fr = {}
    if probe:
        peak = probe["product_peak_per_s"] / 1e12
        lohi = probe["lo_hi_product"]["per_s"] / 1e12
        for name, prods, cnt, t in (("encrypt (2^20)", prod_enc, N_PLAIN, enc_ms), ("decrypt (2^16 aggregates)", prod_dec,
                                    per_group, dec_ms), ("decrypt (2^20 ciphertexts)", prod_dec, N_PLAIN, dec_full_ms),
                                    ("k_hom_sum", prod_sum, per_group, sum_ms)):
            a = prods * cnt / (t / 1e3) / 1e12
            fr[name] = {"achieved_tprod_s": a, "frac_of_measured_peak": a / peak, "frac_of_lo_hi_rate": a / lohi}
        roof = {"bound": "alu", "kernel": "k_enc_crt", "achieved": ach_enc, "peak": peak,
                "unit": "T word products/s (32x32->64)", "frac": ach_enc / peak,
                "peak_note": "measured: pc2_probe_mul %s rate (of measured), the fastest way this GPU forms a "
                             "32x32->64 product; %.0f MHz effective" % (probe["product_peak_kind"],
                                                                        probe[probe["product_peak_kind"]]["sm_mhz"]),
                "nominal": {"peak_timad_s": nominal_imad, "achieved_timad_s": imad_per_elem * N_PLAIN / (enc_ms / 1e3) / 1e12,
                            "note": "%d SMs x %d IMAD/clk x %.0f MHz, hi and lo halves counted as two IMADs" % (
                                sms, IMAD_PER_CLK_SM, sm_max)}}
    else:
        a = imad_per_elem * N_PLAIN / (enc_ms / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": "k_enc_crt", "achieved": a, "peak": nominal_imad, "unit": "TIMAD/s",
                "frac": a / nominal_imad, "peak_note": "nominal (probe skipped): %d SMs x %d IMAD/clk x %.0f MHz" % (
                    sms, IMAD_PER_CLK_SM, sm_max)}
    roof["traffic"] = ENC_DRAM_BYTES_PER_ELEM * N_PLAIN if ENC_DRAM_BYTES_PER_ELEM else None
    if stages and stages["encrypt"] and probe:
        # the dominant kernel of the tensor-core path: the full-width powers
        # (k_modexp_tc).  Its integer pipe forms T = a b (a squaring's cross
        # products and squares: L (L + 1) / 2 word products; a general
        # product: L^2); its tensor cores the reduction's contractions
        # (73728 f16 MACs per product and element).
        sq, mu, lb = pc2.power_counts(key, 0)
        imad_prod = sq * lb * (lb + 1) // 2 + mu * lb * lb
        t_pow = (stages["encrypt"]["power_p2"] + stages["encrypt"]["power_q2"]) / 1e3
        ach = imad_prod * N_PLAIN / t_pow / 1e12
        roww = probe["wide_row_64_limbs"]["per_s"] / 1e12
        tflops = 2.0 * 73728 * (sq + mu) * N_PLAIN / t_pow / 1e12
        cios_eq = (sq + mu) * (2 * lb * lb + lb) * N_PLAIN / t_pow / 1e12
        peak_tc = peaks.get("bf16_tflops")
        roof = {"bound": "alu", "kernel": "k_modexp_tc", "achieved": ach, "peak": roww,
                "unit": "T word products/s (integer pipe: one mad.wide.u32 and a 64-bit add per 32x32->64 product)",
                "frac": ach / roww, "traffic": TC_DRAM_BYTES_PER_ELEM * N_PLAIN if TC_DRAM_BYTES_PER_ELEM else None,
                "peak_note": "measured: pc2_probe_mul wide_row_64_limbs rate (of measured), 64-limb rows in the "
                             "instruction pattern of the kernel's products; achieved over both launches of the "
                             "encryption's powers (mod p^2, q^2), CUDA events on the launching stream",
                "frac_of_mad_wide": ach / (probe["mad_wide"]["per_s"] / 1e12),
                "per_element": {"squarings": sq, "products": mu, "limbs": lb, "integer_pipe_word_products": imad_prod,
                                "tensor_macs": 73728 * (sq + mu)},
                "tensor": {"achieved_tflops": tflops, "peak_tflops": peak_tc,
                           "frac": tflops / peak_tc if peak_tc else None,
                           "peak_note": "MEASURED_PEAKS.json bf16_tflops (f16 and bf16 share the dense rate)"},
                "cios_equivalent": {"achieved": cios_eq, "unit": "T word products/s (2 L^2 + L per Montgomery product)",
                                    "frac_of_mad_wide_peak": cios_eq / (probe["product_peak_per_s"] / 1e12)},
                "launches_s": t_pow}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_bits": NBITS, "plaintexts_per_gpu": N_PLAIN, "groups": GROUPS,
                   "encrypt_path": "key-owner CRT (mod p^2, q^2)", "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": "dp%d (independent shards)" % world},
        "detail": {"encrypt_ms": enc_ms, "hom_sum_ms": sum_ms, "decrypt_ms": dec_ms,
                   "enc_per_s": N_PLAIN / (enc_ms / 1e3), "dec_per_s": per_group / (dec_ms / 1e3),
                   "decrypt_all_2p20_ms": dec_full_ms,
                   "dec_per_s_all_2p20": N_PLAIN / (dec_full_ms / 1e3) if dec_full_ms else None,
                   "enc_montmuls_per_elem": mm, "enc_half_width_montmuls_per_elem": mmh,
                   "dec_montmuls_per_elem": dmm, "montmul_limbs": lb, "enc_imads_per_elem": imad_per_elem,
                   "enc_products_per_elem": prod_enc, "dec_products_per_elem": prod_dec,
                   "hom_sum_products_per_elem": prod_sum, "fractions": fr, "engine_ab": engine_ab,
                   "tc_stages_ms": stages,
                   "engine": {-1: "automatic (tensor cores from %d elements at 2048 bits)" % 16384,
                              0: "integer pipe", 1: "tensor cores"}[args.engine]},
        "multiplier_probe": probe,
        "roofline": roof,
        "e2e": {"value": ops / (ms_e2e / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(m_pinned.numel() * 8),
                "d2h_bytes_per_step": int(dec_host.numel() * 4)},
        "gpu_launches": 3 * args.steps,
        "clocks": clk,
        "cpu_baseline": cpu_base,
        "admm": None if args.no_admm else run_admm(dev),
        "batch": None if args.no_batch else run_batch(dev, args.batch_rounds),
        "serve": None if args.no_serve else run_serve(dev),
        "table2": None if args.no_table2 else run_table2(dev),
        "hbm": None if args.no_hbm else run_hbm(dev, n=args.hbm_elems, n_dec=min(args.hbm_elems, 1 << 24)),
        "admm_full": None if args.no_admm_full else run_admm_full(dev),
        "tc_mont": None if args.no_tc else run_tc_mont(dev),
    }
    if line["hbm"] and probe:
        # the z/v update spends three IEEE double additions per element
        # (v + x, a - kappa, a - z); against the measured FP64 add rate
        zv = line["hbm"]["steps"]["zv_update"]
        rate = probe["fp64_add"]["per_s"]
        zv["fp64_adds_per_elem"] = 3
        zv["fp64_frac"] = 3 * zv["elements"] / (zv["ms"] / 1e3) / rate
        zv["fp64_add_peak_per_s"] = rate
    print(json.dumps(line))
    if dist: dist.destroy_process_group()


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    v, cores, sample, per = _cpu_reference(steps=args.steps, warmup=args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_bits": NBITS, "plaintexts_per_gpu": N_PLAIN, "groups": GROUPS},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pc2", choices=["pc2", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-admm", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-table2", action="store_true", help="skip the Table II operations at 1024/2048/4096 bits")
    ap.add_argument("--no-hbm", action="store_true", help="skip the bandwidth of the memory-bound steps")
    ap.add_argument("--hbm-elems", type=int, default=1 << 27, help="vector length of the bandwidth section")
    ap.add_argument("--no-admm-full", action="store_true", help="skip the full-scale 3072-bit ADMM (about 2 min)")
    ap.add_argument("--no-probe", action="store_true", help="skip the multiplier probe (roofline on the nominal peak)")
    ap.add_argument("--no-tc", action="store_true", help="skip the tensor-core Montgomery experiment")
    ap.add_argument("--engine", type=int, default=-1, choices=[-1, 0, 1],
                    help="full-width powers at 2048 bits: -1 automatic, 0 integer pipe, 1 tensor cores")
    ap.add_argument("--no-engine-ab", action="store_true", help="skip the per-engine encryption/decryption timing")
    ap.add_argument("--tc-only", action="store_true", help="run only the tensor-core Montgomery experiment")
    ap.add_argument("--batch-rounds", type=int, default=1)
    ap.add_argument("--plaintexts", type=int, default=N_PLAIN, help="per GPU (reduced sizes are for profiling only)")
    ap.add_argument("--groups", type=int, default=GROUPS)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.tc_only:
        import torch

        torch.cuda.set_device(0)
        print(json.dumps({"tc_mont": run_tc_mont(0)}))
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
