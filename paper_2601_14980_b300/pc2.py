"""Thin ctypes binding of libpc2 (include/pc2.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Device vectors are torch tensors (int32 for 32-bit words, int64 for
64-bit plaintexts, reinterpreted bit for bit); the library never sees torch
types.  Importing this module raises if libpc2.so is missing -- there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libpc2.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libpc2.so not built (run python -m paper_2601_14980_b300.build): %s" % LIB_PATH)
_lib = ctypes.CDLL(LIB_PATH)

_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64
_i = ctypes.c_int


def _sig(name, args, res=_i):
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = res
    return f


_strerror = _sig("pc2_strerror", [_i], ctypes.c_char_p)
_ctx_create = _sig("pc2_ctx_create", [_i, ctypes.POINTER(_vp)])
_ctx_destroy = _sig("pc2_ctx_destroy", [_vp], None)
_ctx_reserve = _sig("pc2_ctx_reserve", [_vp, _sz])
_ctx_scratch_bytes = _sig("pc2_ctx_scratch_bytes", [_vp], _sz)
_ctx_status = _sig("pc2_ctx_status", [_vp, _vp, ctypes.POINTER(_i)])
_ctx_set_window = _sig("pc2_ctx_set_window", [_vp, _i])
_keygen = _sig("pc2_keygen", [_i, _u64, ctypes.POINTER(_vp)])
_key_from_primes = _sig("pc2_key_from_primes", [_vp, _vp, _i, ctypes.POINTER(_vp)])
_key_public = _sig("pc2_key_public", [_vp, ctypes.POINTER(_vp)])
_key_destroy = _sig("pc2_key_destroy", [_vp], None)
_key_info = _sig("pc2_key_info", [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i)])
_key_export = _sig("pc2_key_export", [_vp, _vp, _vp, _vp, _vp, _vp])
_key_cost = _sig("pc2_key_cost", [_vp, _vp, _i, ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_long),
                                    ctypes.POINTER(_i)])
_tiled_words = _sig("pc2_tiled_words", [_sz, _i], _sz)
_pack = _sig("pc2_pack", [_vp, _vp, _sz, _i, _vp, _vp])
_unpack = _sig("pc2_unpack", [_vp, _vp, _sz, _i, _vp, _vp])
_encrypt = _sig("pc2_encrypt", [_vp, _vp, _vp, _sz, _u64, _u32, _u64, _vp, _vp])
_encrypt_wide = _sig("pc2_encrypt_wide", [_vp, _vp, _vp, _sz, _u64, _u32, _u64, _vp, _vp])
_encrypt_public = _sig("pc2_encrypt_public", [_vp, _vp, _vp, _sz, _u64, _u32, _u64, _vp, _vp])
_decrypt = _sig("pc2_decrypt", [_vp, _vp, _vp, _sz, _vp, _vp])
_hom_add = _sig("pc2_hom_add", [_vp, _vp, _vp, _vp, _sz, _vp, _vp])
_hom_sum = _sig("pc2_hom_sum", [_vp, _vp, _vp, _sz, _sz, _vp, _vp])
_hom_scal = _sig("pc2_hom_scal", [_vp, _vp, _vp, _vp, _sz, _vp, _vp])
_hom_scal_wide = _sig("pc2_hom_scal_wide", [_vp, _vp, _vp, _vp, _sz, _vp, _vp])

ST_RANGE, ST_QUANT, ST_TIMEOUT = 1, 2, 4
OK, EINVAL, ERANGE, EKEY, ENOMEM, ECUDA, ETIMEOUT, EMISSING, EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7, -8
COST_ENCRYPT, COST_ENCRYPT_PUBLIC, COST_DECRYPT = 0, 1, 2  # pc2_key_cost operations


class Pc2Error(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__("%s: %s (%d)" % (what, _strerror(code).decode(), code))
        self.code = code


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise Pc2Error(rc, what)


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def _stream(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def tiled_words(count: int, limbs: int) -> int:
    return int(_tiled_words(count, limbs))


class Context:
    """A library context on one CUDA device (scratch memory, status word)."""

    def __init__(self, device: int = 0):
        h = _vp()
        _check(_ctx_create(device, ctypes.byref(h)), "pc2_ctx_create")
        self.h = h
        self.device = device

    def close(self):
        if self.h:
            _ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reserve(self, nbytes: int):
        _check(_ctx_reserve(self.h, nbytes), "pc2_ctx_reserve")

    @property
    def scratch_bytes(self) -> int:
        return int(_ctx_scratch_bytes(self.h))

    def status(self, stream=None) -> int:
        bits = _i()
        _check(_ctx_status(self.h, _stream(stream), ctypes.byref(bits)), "pc2_ctx_status")
        return bits.value

    def set_window(self, w: int):
        _check(_ctx_set_window(self.h, w), "pc2_ctx_set_window")


def _words_of(x: int, nw: int) -> np.ndarray:
    return np.frombuffer(int(x).to_bytes(4 * nw, "little"), dtype=np.uint32).copy()


def _int_of(w: np.ndarray) -> int:
    return int.from_bytes(np.ascontiguousarray(w, dtype=np.uint32).tobytes(), "little")


class Key:
    """A Paillier key held by the library (host)."""

    def __init__(self, handle):
        self.h = handle
        nb, pv = _i(), _i()
        _check(_key_info(self.h, ctypes.byref(nb), ctypes.byref(pv)), "pc2_key_info")
        self.nbits = nb.value
        self.has_private = bool(pv.value)

    @classmethod
    def generate(cls, nbits: int, seed: int) -> "Key":
        h = _vp()
        _check(_keygen(nbits, seed, ctypes.byref(h)), "pc2_keygen")
        return cls(h)

    @classmethod
    def from_primes(cls, p: int, q: int) -> "Key":
        nw = max((p.bit_length() + 31) // 32, (q.bit_length() + 31) // 32)
        pa, qa = _words_of(p, nw), _words_of(q, nw)
        h = _vp()
        _check(_key_from_primes(pa.ctypes.data, qa.ctypes.data, nw, ctypes.byref(h)), "pc2_key_from_primes")
        return cls(h)

    def public(self) -> "Key":
        h = _vp()
        _check(_key_public(self.h, ctypes.byref(h)), "pc2_key_public")
        return Key(h)

    def close(self):
        if self.h:
            _key_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def limbs(self) -> int:
        return self.nbits // 32

    def export(self) -> dict:
        L = self.limbs
        n = np.zeros(L, np.uint32)
        if not self.has_private:
            _check(_key_export(self.h, n.ctypes.data, None, None, None, None), "pc2_key_export")
            return {"n": _int_of(n)}
        p, q = np.zeros(L // 2, np.uint32), np.zeros(L // 2, np.uint32)
        lam, mu = np.zeros(L, np.uint32), np.zeros(L, np.uint32)
        _check(_key_export(self.h, n.ctypes.data, p.ctypes.data, q.ctypes.data, lam.ctypes.data, mu.ctypes.data),
               "pc2_key_export")
        return {"n": _int_of(n), "p": _int_of(p), "q": _int_of(q), "lambda": _int_of(lam), "mu": _int_of(mu)}

    def cost(self, ctx: Context, op: int) -> tuple[int, int, int]:
        """(Montgomery products per element of `limbs` words, those of limbs/2
        words, limbs) of one op."""
        mm, mh, lb = ctypes.c_long(), ctypes.c_long(), _i()
        _check(_key_cost(ctx.h, self.h, op, ctypes.byref(mm), ctypes.byref(mh), ctypes.byref(lb)), "pc2_key_cost")
        return mm.value, mh.value, lb.value

    def products(self, ctx: Context, op: int) -> int:
        """Algorithmic 32x32->64 word products per element of one op's powers:
        a Montgomery product of L limbs takes 2 L^2 + L (the L^2 limb products
        of a*b and of m*N, and L quotient words)."""
        mm, mh, lb = self.cost(ctx, op)
        h = lb // 2
        return mm * (2 * lb * lb + lb) + mh * (2 * h * h + h)

    def imads(self, ctx: Context, op: int) -> int:
        """Algorithmic 32-bit multiply-adds per element of one op's powers: a
        Montgomery product of L limbs takes 4 L^2 + L (low and high halves of
        the L^2 limb products of a*b and of m*N, and L quotient words)."""
        mm, mh, lb = self.cost(ctx, op)
        h = lb // 2
        return mm * (4 * lb * lb + lb) + mh * (4 * h * h + h)


# ------------------------------------------------------------------ device buffers
def empty_tiled(count: int, limbs: int, device="cuda"):
    import torch

    return torch.empty(max(tiled_words(count, limbs), 1), dtype=torch.int32, device=device)


def pack(ctx: Context, canon, count: int, limbs: int, out=None, stream=None):
    out = empty_tiled(count, limbs, canon.device) if out is None else out
    _check(_pack(ctx.h, _ptr(canon), count, limbs, _ptr(out), _stream(stream)), "pc2_pack")
    return out


def unpack(ctx: Context, tiled, count: int, limbs: int, out=None, stream=None):
    import torch

    out = torch.empty(max(count * limbs, 1), dtype=torch.int32, device=tiled.device) if out is None else out
    _check(_unpack(ctx.h, _ptr(tiled), count, limbs, _ptr(out), _stream(stream)), "pc2_unpack")
    return out


def ints_to_tiled(ctx: Context, values: Sequence[int], limbs: int, device="cuda"):
    """Python ints -> canonical words on the host -> device -> tiled (marshalling)."""
    import torch

    canon = np.concatenate([_words_of(v, limbs) for v in values]) if len(values) else np.zeros(1, np.uint32)
    d = torch.from_numpy(canon.view(np.int32)).to(device)
    return pack(ctx, d, len(values), limbs)


def tiled_to_ints(ctx: Context, tiled, count: int, limbs: int) -> list[int]:
    import torch

    canon = unpack(ctx, tiled, count, limbs)
    torch.cuda.synchronize()
    w = canon.cpu().numpy().view(np.uint32)
    return [_int_of(w[i * limbs:(i + 1) * limbs]) for i in range(count)]


# ------------------------------------------------------------------ Paillier
def encrypt(ctx: Context, key: Key, m, seed: int, stream_id: int, e0: int = 0, out=None, public: bool = False,
            stream=None):
    """Eq. (itq1) on `m` (int64 tensor of uint64 plaintexts).  Returns tiled ciphertexts."""
    count = int(m.numel())
    out = empty_tiled(count, 2 * key.limbs, m.device) if out is None else out
    fn = _encrypt_public if public else _encrypt
    _check(fn(ctx.h, key.h, _ptr(m), count, seed, stream_id, e0, _ptr(out), _stream(stream)), "pc2_encrypt")
    return out


def encrypt_wide(ctx: Context, key: Key, m_tiled, count: int, seed: int, stream_id: int, e0: int = 0, out=None,
                 stream=None):
    out = empty_tiled(count, 2 * key.limbs, m_tiled.device) if out is None else out
    _check(_encrypt_wide(ctx.h, key.h, _ptr(m_tiled), count, seed, stream_id, e0, _ptr(out), _stream(stream)),
           "pc2_encrypt_wide")
    return out


def decrypt(ctx: Context, key: Key, ct, count: int, out=None, stream=None):
    """Sec. III-C decryption; returns tiled plaintexts of key.limbs words."""
    out = empty_tiled(count, key.limbs, ct.device) if out is None else out
    _check(_decrypt(ctx.h, key.h, _ptr(ct), count, _ptr(out), _stream(stream)), "pc2_decrypt")
    return out


def hom_add(ctx: Context, key: Key, a, b, count: int, out=None, stream=None):
    out = empty_tiled(count, 2 * key.limbs, a.device) if out is None else out
    _check(_hom_add(ctx.h, key.h, _ptr(a), _ptr(b), count, _ptr(out), _stream(stream)), "pc2_hom_add")
    return out


def hom_sum(ctx: Context, key: Key, ct_groups, groups: int, count: int, out=None, stream=None):
    out = empty_tiled(count, 2 * key.limbs, ct_groups.device) if out is None else out
    _check(_hom_sum(ctx.h, key.h, _ptr(ct_groups), groups, count, _ptr(out), _stream(stream)), "pc2_hom_sum")
    return out


def hom_scal(ctx: Context, key: Key, ct, k, count: int, out=None, stream=None):
    out = empty_tiled(count, 2 * key.limbs, ct.device) if out is None else out
    _check(_hom_scal(ctx.h, key.h, _ptr(ct), _ptr(k), count, _ptr(out), _stream(stream)), "pc2_hom_scal")
    return out


def hom_scal_wide(ctx: Context, key: Key, ct, k, count: int, out=None, stream=None):
    """c_i^{k_i} mod n^2 with k a tiled array of full-width scalars (nbits/32 limbs)."""
    out = empty_tiled(count, 2 * key.limbs, ct.device) if out is None else out
    _check(_hom_scal_wide(ctx.h, key.h, _ptr(ct), _ptr(k), count, _ptr(out), _stream(stream)), "pc2_hom_scal_wide")
    return out


# ------------------------------------------------------------------ quantizer and ADMM
_quantize = _sig("pc2_quantize", [_vp, _vp, _sz, ctypes.c_double, ctypes.c_double, _i, _i, _i, _vp, _vp])


class _AdmmParams(ctypes.Structure):
    _fields_ = [("nodes", _i), ("node_sizes", ctypes.POINTER(_i)), ("lambda_", ctypes.c_double),
                ("rho", ctypes.c_double), ("zmin", ctypes.c_double), ("zmax", ctypes.c_double),
                ("log2_scale", _i), ("seed", _u64), ("per_node", _i)]


_admm_create = _sig("pc2_admm_create", [_vp, _vp, ctypes.POINTER(_AdmmParams), _vp, _vp, ctypes.POINTER(_vp), _vp])
_admm_destroy = _sig("pc2_admm_destroy", [_vp], None)
_admm_reset = _sig("pc2_admm_reset", [_vp, _vp])
_admm_round = _sig("pc2_admm_round", [_vp, _i, _vp])
_admm_set_node_present = _sig("pc2_admm_set_node_present", [_vp, _i, _i])
_admm_round_plain = _sig("pc2_admm_round_plain", [_vp, _i, _vp])
_admm_get = _sig("pc2_admm_get", [_vp, _vp, _vp, _vp, ctypes.POINTER(_u32), _vp])
_admm_set = _sig("pc2_admm_set", [_vp, _vp, _vp, _vp, _u32, _vp])
_admm_buffers = _sig("pc2_admm_buffers", [_vp] + [ctypes.POINTER(_vp)] * 5 + [ctypes.POINTER(_i)])
_admm_set_matvec = _sig("pc2_admm_set_matvec", [_vp, _i])
_admm_info = _sig("pc2_admm_info", [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i)])


def quantize(ctx: Context, u, zmin: float, zmax: float, log2_scale: int, gamma: int = 2, negate: bool = False,
             out=None, stream=None):
    """Eq. (et21) on a float64 tensor; returns an int64 tensor of uint64 codes."""
    import torch

    out = torch.empty(u.numel(), dtype=torch.int64, device=u.device) if out is None else out
    _check(_quantize(ctx.h, _ptr(u), u.numel(), zmin, zmax, log2_scale, gamma, int(negate), _ptr(out),
                     _stream(stream)), "pc2_quantize")
    return out


class Admm:
    """Algorithm 1 of the paper on one GPU (see include/pc2.h)."""

    def __init__(self, ctx: Context, key: Key, node_sizes, alpha, Bbar, lam: float, rho: float, zmin: float,
                 zmax: float, log2_scale: int, seed: int, per_node: bool = False, stream=None):
        sizes = (_i * len(node_sizes))(*[int(s) for s in node_sizes])
        self._sizes = sizes
        p = _AdmmParams(len(node_sizes), sizes, lam, rho, zmin, zmax, log2_scale, seed, int(per_node))
        h = _vp()
        _check(_admm_create(ctx.h, key.h, ctypes.byref(p), _ptr(alpha), _ptr(Bbar), ctypes.byref(h), _stream(stream)),
               "pc2_admm_create")
        self.h = h
        self.N = int(sum(node_sizes))
        self.ctx, self.key = ctx, key

    def close(self):
        if self.h:
            _admm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self, stream=None):
        _check(_admm_reset(self.h, _stream(stream)), "pc2_admm_reset")

    def round(self, rounds: int = 1, stream=None):
        _check(_admm_round(self.h, rounds, _stream(stream)), "pc2_admm_round")

    def round_plain(self, rounds: int = 1, stream=None):
        _check(_admm_round_plain(self.h, rounds, _stream(stream)), "pc2_admm_round_plain")

    def set_node_present(self, node: int, present: bool):
        """Marks edge node `node`'s segment as arrived or missing (pc2_admm_set_node_present)."""
        _check(_admm_set_node_present(self.h, int(node), int(bool(present))), "pc2_admm_set_node_present")

    def get(self, stream=None):
        import torch

        x, z, v = (torch.empty(self.N, dtype=torch.float64, device="cuda") for _ in range(3))
        r = _u32()
        _check(_admm_get(self.h, _ptr(x), _ptr(z), _ptr(v), ctypes.byref(r), _stream(stream)), "pc2_admm_get")
        return x, z, v, r.value

    def set(self, x, z, v, round_: int, stream=None):
        _check(_admm_set(self.h, _ptr(x), _ptr(z), _ptr(v), round_, _stream(stream)), "pc2_admm_set")

    def buffers(self) -> dict:
        ps = [_vp() for _ in range(5)]
        n = _i()
        _check(_admm_buffers(self.h, *[ctypes.byref(p) for p in ps], ctypes.byref(n)), "pc2_admm_buffers")
        return dict(zip(["zhat", "vhat", "xhat", "alpha_hat", "D"], [p.value for p in ps]), N=n.value)

    def save(self):
        """Host checkpoint: (x, z, v) as numpy arrays and the next round."""
        x, z, v = (np.empty(self.N, dtype=np.float64) for _ in range(3))
        r = _u32()
        _check(_admm_save(self.h, x.ctypes.data, z.ctypes.data, v.ctypes.data, ctypes.byref(r)), "pc2_admm_save")
        return x, z, v, r.value

    def load(self, x, z, v, round_: int):
        x, z, v = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, z, v))
        _check(_admm_load(self.h, x.ctypes.data, z.ctypes.data, v.ctypes.data, round_), "pc2_admm_load")

    def set_matvec(self, mode: int):
        """0 automatic, 1 one CTA per row tile, 2 bucket windows spread over CTAs."""
        _check(_admm_set_matvec(self.h, mode), "pc2_admm_set_matvec")

    def info(self) -> dict:
        c, nw, nt = _i(), _i(), _i()
        _check(_admm_info(self.h, ctypes.byref(c), ctypes.byref(nw), ctypes.byref(nt)), "pc2_admm_info")
        return {"c": c.value, "nwin": nw.value, "ntiles": nt.value}


def device_words(ptr: int, nwords: int, device="cuda"):
    """A torch view-copy of `nwords` 32-bit words at a library-owned device pointer (for tests)."""
    import torch

    out = torch.empty(nwords, dtype=torch.int32, device=device)
    torch.cuda.synchronize()
    _lib_copy(out.data_ptr(), ptr, nwords * 4)
    return out


def _lib_copy(dst: int, src: int, nbytes: int):
    import torch

    # torch has no raw-pointer view; use cudaMemcpy through the CUDA runtime torch links against
    rt = ctypes.CDLL(_cudart_path())
    rt.cudaMemcpy.argtypes = [_vp, _vp, _sz, _i]
    rt.cudaMemcpy.restype = _i
    if rt.cudaMemcpy(dst, src, nbytes, 3) != 0:  # cudaMemcpyDeviceToDevice
        raise RuntimeError("cudaMemcpy failed")
    torch.cuda.synchronize()


def _cudart_path() -> str:
    import glob as _g

    import torch

    cands = _g.glob(os.path.join(os.path.dirname(torch.__file__), "lib", "libcudart*.so*"))
    cands += _g.glob("/usr/local/cuda/lib64/libcudart.so*")
    if not cands:
        raise RuntimeError("libcudart not found")
    return cands[0]


_ctx_set_lanes = _sig("pc2_ctx_set_lanes", [_vp, _i])
_autotune = _sig("pc2_autotune", [_vp, _vp, _sz, _i, _vp, ctypes.POINTER(_i)])


def set_lanes(ctx: Context, lanes: int):
    """Force lanes per element (1, 2, 4, 8) where built; 0 = automatic."""
    _check(_ctx_set_lanes(ctx.h, lanes), "pc2_ctx_set_lanes")


def autotune(ctx: Context, key: Key, count: int, encrypt: bool = True, decrypt: bool = True, stream=None) -> dict:
    """Run the library's autotuner for `count`-element calls; returns the chosen (lanes, window, split) per op."""
    ops = (1 if encrypt else 0) | (2 if decrypt else 0)
    res = (_i * 6)()
    _check(_autotune(ctx.h, key.h, count, ops, _stream(stream), res), "pc2_autotune")
    out, i = {}, 0
    if encrypt:
        out["encrypt"] = (res[0], res[1], res[2])
        i = 3
    if decrypt:
        out["decrypt"] = (res[i], res[i + 1], res[i + 2])
    return out


_ctx_set_split = _sig("pc2_ctx_set_split", [_vp, _i])


_set_engine = _sig("pc2_ctx_set_engine", [_vp, _i])


def set_engine(ctx: Context, engine: int):
    """Full-width powers at 2048-bit n: -1 automatic, ENGINE_IMAD, ENGINE_TC (pc2_ctx_set_engine)."""
    _check(_set_engine(ctx.h, engine), "pc2_ctx_set_engine")


_set_timing = _sig("pc2_ctx_set_timing", [_vp, _i])
_stage_ms = _sig("pc2_ctx_stage_ms", [_vp, ctypes.POINTER(ctypes.c_double)])
_power_counts = _sig("pc2_key_power_counts", [_vp, _i, ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_long),
                                              ctypes.POINTER(_i)])


def set_timing(ctx: Context, on: bool):
    _check(_set_timing(ctx.h, int(on)), "pc2_ctx_set_timing")


def stage_ms(ctx: Context) -> list:
    """[set-up, power mod p^2, power mod q^2, finish] of the last timed tensor-core call (ms)."""
    out = (ctypes.c_double * 4)()
    _check(_stage_ms(ctx.h, out), "pc2_ctx_stage_ms")
    return list(out)


def power_counts(key: Key, op: int) -> tuple:
    """(squarings, products, limbs) of the full-width powers of one element's op (0 encrypt, 2 decrypt)."""
    sq, mu, lb = ctypes.c_long(), ctypes.c_long(), _i()
    _check(_power_counts(key.h, op, ctypes.byref(sq), ctypes.byref(mu), ctypes.byref(lb)), "pc2_key_power_counts")
    return sq.value, mu.value, lb.value


def set_split(ctx: Context, mode: int):
    """CRT halves in parallel: 0 automatic, 1 never, 2 always."""
    _check(_ctx_set_split(ctx.h, mode), "pc2_ctx_set_split")


class _BatchParams(ctypes.Structure):
    _fields_ = [("nodes", _i), ("node_sizes", ctypes.POINTER(_i)), ("node_key", ctypes.POINTER(_i)),
                ("nkeys", _i), ("keys", ctypes.POINTER(_vp)), ("lambda_", ctypes.c_double),
                ("rho", ctypes.c_double), ("zmin", ctypes.c_double), ("zmax", ctypes.c_double),
                ("log2_scale", _i), ("seed", _u64)]


_batch_create = _sig("pc2_batch_create", [_vp, ctypes.POINTER(_BatchParams), _vp, _vp, ctypes.POINTER(_vp), _vp])
_batch_destroy = _sig("pc2_batch_destroy", [_vp], None)
_batch_reset = _sig("pc2_batch_reset", [_vp, _vp])
_batch_round = _sig("pc2_batch_round", [_vp, _i, _vp])
_batch_round_per_node = _sig("pc2_batch_round_per_node", [_vp, _i, _vp])
_batch_get = _sig("pc2_batch_get", [_vp, _vp, _vp, _vp, ctypes.POINTER(_u32), _vp])
_batch_ciphertexts = _sig("pc2_batch_ciphertexts", [_vp, _i, _i, ctypes.POINTER(_vp), ctypes.POINTER(_i)])
_batch_info = _sig("pc2_batch_info", [_vp, ctypes.POINTER(_sz), ctypes.POINTER(_i), ctypes.POINTER(_i),
                                      ctypes.POINTER(_sz)])
_batch_tune = _sig("pc2_batch_tune", [_vp, _i, _vp, ctypes.POINTER(_i)])


class Batch:
    """Batched rounds over many edge nodes with mixed key sizes (see include/pc2.h)."""

    def __init__(self, ctx: Context, keys, node_sizes, node_key, alpha, bdiag, lam: float, rho: float, zmin: float,
                 zmax: float, log2_scale: int, seed: int, stream=None):
        K = len(node_sizes)
        self._sizes = (_i * K)(*[int(s) for s in node_sizes])
        self._nkey = (_i * K)(*[int(s) for s in node_key])
        self._keys = (_vp * len(keys))(*[k.h for k in keys])
        p = _BatchParams(K, self._sizes, self._nkey, len(keys), self._keys, lam, rho, zmin, zmax, log2_scale, seed)
        h = _vp()
        _check(_batch_create(ctx.h, ctypes.byref(p), _ptr(alpha), _ptr(bdiag), ctypes.byref(h), _stream(stream)),
               "pc2_batch_create")
        self.h = h
        self.N = int(sum(node_sizes))
        self.ctx, self.keys = ctx, keys

    def close(self):
        if self.h:
            _batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self, stream=None):
        _check(_batch_reset(self.h, _stream(stream)), "pc2_batch_reset")

    def round(self, rounds: int = 1, stream=None):
        _check(_batch_round(self.h, rounds, _stream(stream)), "pc2_batch_round")

    def round_per_node(self, rounds: int = 1, stream=None):
        _check(_batch_round_per_node(self.h, rounds, _stream(stream)), "pc2_batch_round_per_node")

    def get(self, stream=None):
        import torch

        x, z, v = (torch.empty(self.N, dtype=torch.float64, device="cuda") for _ in range(3))
        r = _u32()
        _check(_batch_get(self.h, _ptr(x), _ptr(z), _ptr(v), ctypes.byref(r), _stream(stream)), "pc2_batch_get")
        return x, z, v, r.value

    def ciphertexts(self, which: str, node: int):
        """(device pointer, limbs) of node `node`'s tiled ciphertexts: alpha_hat, zhat, vhat or xhat."""
        p, limbs = _vp(), _i()
        w = ["alpha_hat", "zhat", "vhat", "xhat"].index(which)
        _check(_batch_ciphertexts(self.h, w, node, ctypes.byref(p), ctypes.byref(limbs)), "pc2_batch_ciphertexts")
        return p.value, limbs.value

    def info(self) -> dict:
        n, it, g, sb = _sz(), _i(), _i(), _sz()
        _check(_batch_info(self.h, ctypes.byref(n), ctypes.byref(it), ctypes.byref(g), ctypes.byref(sb)),
               "pc2_batch_info")
        return {"elements": n.value, "items": it.value, "grid": g.value, "scratch_bytes": sb.value}

    def tune(self, sample_items: int = 0, stream=None) -> dict:
        res = (_i * 6)()
        _check(_batch_tune(self.h, sample_items, _stream(stream), res), "pc2_batch_tune")
        return {"window": {b: res[i] for i, b in enumerate((256, 512, 1024, 2048, 3072)) if res[i]},
                "ctas_per_sm": res[5]}


class _ServerParams(ctypes.Structure):
    _fields_ = [("arena_bytes", _sz), ("mode", _i), ("max_active", _i), ("small_request", _sz),
                ("step_budget", ctypes.c_double)]


_server_create = _sig("pc2_server_create", [_vp, _vp, ctypes.POINTER(_ServerParams), ctypes.POINTER(_vp)])
_server_destroy = _sig("pc2_server_destroy", [_vp], None)
_server_submit = _sig("pc2_server_submit", [_vp, _i, _vp, _sz, _i, _sz, _u64, _u32, _u64, _vp, ctypes.POINTER(_u64)])
_server_wait = _sig("pc2_server_wait", [_vp, _u64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)])
_server_stats = _sig("pc2_server_stats", [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64), ctypes.POINTER(_u64),
                                          ctypes.POINTER(_sz)])

OP_ENCRYPT, OP_DECRYPT, OP_AGGREGATE = 1, 2, 3


class Server:
    """Request loop with continuous batching (mode 0) or the plain per-request path (mode 1)."""

    def __init__(self, ctx: Context, key: Key, arena_bytes: int, mode: int = 0, max_active: int = 0,
                 small_request: int = 0, step_budget: float = 0.0):
        p = _ServerParams(arena_bytes, mode, max_active, small_request, step_budget)
        h = _vp()
        _check(_server_create(ctx.h, key.h, ctypes.byref(p), ctypes.byref(h)), "pc2_server_create")
        self.h = h
        self.key = key
        self._keep = {}

    def close(self):
        if self.h:
            _server_destroy(self.h)
            self.h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, op: int, h_in, count: int, h_out, groups: int = 1, seed: int = 0, stream: int = 0,
               e0: int = 0, h_stride: int = 0) -> int:
        """h_in / h_out: host torch tensors (page-locked for overlap), kept alive until wait()."""
        t = _u64()
        _check(_server_submit(self.h, op, h_in.data_ptr(), count, groups, h_stride, seed, stream, e0,
                              h_out.data_ptr(), ctypes.byref(t)), "pc2_server_submit")
        self._keep[t.value] = (h_in, h_out)
        return t.value

    def wait(self, ticket: int, timeout: float = 600.0) -> float:
        lat = ctypes.c_double()
        rc = _server_wait(self.h, ticket, timeout, ctypes.byref(lat))
        if rc != -6:  # PC2_ETIMEOUT keeps the ticket
            self._keep.pop(ticket, None)
        _check(rc, "pc2_server_wait")
        return lat.value

    def stats(self) -> dict:
        c, s, i, a = _u64(), _u64(), _u64(), _sz()
        _check(_server_stats(self.h, ctypes.byref(c), ctypes.byref(s), ctypes.byref(i), ctypes.byref(a)),
               "pc2_server_stats")
        return {"completed": c.value, "steps": s.value, "items": i.value, "arena_peak": a.value}


_dequantize = _sig("pc2_dequantize", [_vp, _vp, _sz, ctypes.c_double, _i, _i, _vp, _vp])
_zv_update = _sig("pc2_zv_update", [_vp, _vp, _vp, _vp, _sz, ctypes.c_double, _vp])
_decode_matvec = _sig("pc2_decode_matvec", [_vp, _vp, _i, _sz, _vp, _vp, _vp, ctypes.c_double, _i, _vp, _vp])
_hom_matvec = _sig("pc2_hom_matvec", [_vp, _vp, _vp, _vp, _vp, _sz, _i, _vp, _vp])
_admm_save = _sig("pc2_admm_save", [_vp, _vp, _vp, _vp, ctypes.POINTER(_u32)])
_admm_load = _sig("pc2_admm_load", [_vp, _vp, _vp, _vp, _u32])


def zv_update(ctx: Context, x, z, v, kappa: float, stream=None):
    """Eqs. (ty32), (u78) in place on float64 tensors: z = S_kappa(v + x), v = v + x - z."""
    n = int(x.numel())
    _check(_zv_update(ctx.h, _ptr(x), _ptr(z), _ptr(v), n, kappa, _stream(stream)), "pc2_zv_update")


def dequantize(ctx: Context, q, zmin: float, log2_scale: int, gamma: int = 2, out=None, stream=None):
    """Inverse of quantize: q (int64 tensor of uint64) -> float64 tensor."""
    import torch

    n = int(q.numel())
    out = torch.empty(n, dtype=torch.float64, device=q.device) if out is None else out
    _check(_dequantize(ctx.h, _ptr(q), n, zmin, log2_scale, gamma, _ptr(out), _stream(stream)), "pc2_dequantize")
    return out


def decode_matvec(ctx: Context, D, limbs: int, n: int, brow, asum, nk, zmin: float, log2_scale: int, out=None,
                  stream=None):
    """Theorem 1's exact decode of decrypted matvec rows (D tiled, brow int64, asum uint64 as int64, nk int32)."""
    import torch

    out = torch.empty(n, dtype=torch.float64, device=D.device) if out is None else out
    _check(_decode_matvec(ctx.h, _ptr(D), limbs, n, _ptr(brow), _ptr(asum), _ptr(nk), zmin, log2_scale, _ptr(out),
                          _stream(stream)), "pc2_decode_matvec")
    return out


def hom_matvec(ctx: Context, key: Key, alpha, s, K, n: int, kbits: int = 0, out=None, stream=None):
    """Eq. (itq2) on one n x n block (K: int32 tensor of uint32, row-major)."""
    out = empty_tiled(n, 2 * key.limbs, s.device) if out is None else out
    _check(_hom_matvec(ctx.h, key.h, _ptr(alpha), _ptr(s), _ptr(K), n, kbits, _ptr(out), _stream(stream)),
           "pc2_hom_matvec")
    return out


# ------------------------------------------------------------------ multiplier probe
PROBE_LO, PROBE_HI, PROBE_WIDE, PROBE_LOHI, PROBE_ROW, PROBE_DADD, PROBE_ROWW = 0, 1, 2, 3, 4, 5, 6
_probe_mul = _sig("pc2_probe_mul", [_i, _i, _i, _i, _vp, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(_i)])


def probe_mul(device: int, kind: int, blocks_per_sm: int, iters: int, stream=None) -> dict:
    """Throughput of one kind of 32-bit multiply (pc2_probe_mul): operations
    executed, CUDA-event milliseconds, the longest CTA's cycles, SM count."""
    ops, ms, cyc, sms = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), _i()
    _check(_probe_mul(device, kind, blocks_per_sm, iters, _stream(stream), ctypes.byref(ops), ctypes.byref(ms),
                      ctypes.byref(cyc), ctypes.byref(sms)), "pc2_probe_mul")
    return {"ops": ops.value, "ms": ms.value, "cycles": cyc.value, "sms": sms.value}


# ------------------------------------------------------------------ tensor-core Montgomery experiment
ENGINE_IMAD, ENGINE_TC = 0, 1
_mont_sqr = _sig("pc2_mont_sqr", [_vp, _vp, _i, _vp, _sz, _i, _i, _vp, _vp])


def mont_sqr(ctx: Context, n: int, x_tiled, count: int, nsq: int, engine: int, out=None, stream=None):
    """nsq Montgomery squarings mod n (64 words) of a tiled vector (pc2_mont_sqr)."""
    limbs = max(1, (n.bit_length() + 31) // 32)
    nw = _words_of(n, limbs)
    out = empty_tiled(count, limbs, x_tiled.device) if out is None else out
    _check(_mont_sqr(ctx.h, nw.ctypes.data, limbs, _ptr(x_tiled), count, nsq, engine, _ptr(out), _stream(stream)),
           "pc2_mont_sqr")
    return out


# ------------------------------------------------------------------ collaborative CRT split (Algorithm 3)
_collab_mask = _sig("pc2_collab_mask", [_vp, _vp, _vp, _vp, _sz, _vp, _vp])
_collab_edge_encrypt = _sig("pc2_collab_edge_encrypt", [_vp, _vp, _vp, _sz, _u64, _u32, _u64, _vp, _vp])
_collab_master_encrypt = _sig("pc2_collab_master_encrypt", [_vp, _vp, _vp, _vp, _vp, _sz, _u64, _u32, _u64, _vp, _vp])
_collab_edge_reduce = _sig("pc2_collab_edge_reduce", [_vp, _vp, _vp, _sz, _vp, _vp])
_collab_master_decrypt = _sig("pc2_collab_master_decrypt", [_vp, _vp, _vp, _vp, _sz, _vp, _vp])


def collab_mask(ctx: Context, key: Key, w, kappa, count: int, out=None, stream=None):
    out = empty_tiled(count, key.limbs, w.device) if out is None else out
    _check(_collab_mask(ctx.h, key.h, _ptr(w), _ptr(kappa), count, _ptr(out), _stream(stream)), "pc2_collab_mask")
    return out


def collab_edge_encrypt(ctx: Context, key: Key, ow, count: int, seed: int, stream_id: int, e0: int = 0, out=None,
                        stream=None):
    out = empty_tiled(count, key.limbs, ow.device) if out is None else out
    _check(_collab_edge_encrypt(ctx.h, key.h, _ptr(ow), count, seed, stream_id, e0, _ptr(out), _stream(stream)),
           "pc2_collab_edge_encrypt")
    return out


def collab_master_encrypt(ctx: Context, key: Key, w, kappa, cp, count: int, seed: int, stream_id: int, e0: int = 0,
                          out=None, stream=None):
    out = empty_tiled(count, 2 * key.limbs, w.device) if out is None else out
    _check(_collab_master_encrypt(ctx.h, key.h, _ptr(w), _ptr(kappa), _ptr(cp), count, seed, stream_id, e0, _ptr(out),
                                  _stream(stream)), "pc2_collab_master_encrypt")
    return out


def collab_edge_reduce(ctx: Context, key: Key, ct, count: int, out=None, stream=None):
    out = empty_tiled(count, key.limbs, ct.device) if out is None else out
    _check(_collab_edge_reduce(ctx.h, key.h, _ptr(ct), count, _ptr(out), _stream(stream)), "pc2_collab_edge_reduce")
    return out


def collab_master_decrypt(ctx: Context, key: Key, ct, cp, count: int, out=None, stream=None):
    out = empty_tiled(count, key.limbs, ct.device) if out is None else out
    _check(_collab_master_decrypt(ctx.h, key.h, _ptr(ct), _ptr(cp), count, _ptr(out), _stream(stream)),
           "pc2_collab_master_decrypt")
    return out
