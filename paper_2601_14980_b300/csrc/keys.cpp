// keys.cpp -- key generation and the per-key constants of libpc2 (host).
//
// Sec. III-B of the paper: n = pq, epsilon = lambda = lcm(p-1, q-1), g in
// Z*_{n^2} (here g = n + 1), mu = L(g^lambda mod n^2)^-1 mod n with
// L(x) = (x-1)/n; for g = n + 1, L(g^lambda mod n^2) = lambda mod n.
// Everything else here is derived constants for the kernels: Montgomery
// constants of p^2, q^2, n^2, p, q; the exponents n mod p(p-1), n mod q(q-1)
// (Lemma 1: exponents reduce mod phi(p^2) = p(p-1)); (p^2)^-1 mod q^2 for
// Eq. (gA-C-B); h_p = (-q)^-1 mod p, h_q = (-p)^-1 mod q for the CRT
// decryption; and the sliding-window schedules of every fixed exponent.
#include "keys.hpp"

#include <cstring>
#include <memory>
#include <new>

#include "../../include/pc2.h"
#include "philox.h"

namespace pc2 {

bool supported_nbits(int nbits) {
  return nbits == 256 || nbits == 512 || nbits == 1024 || nbits == 2048 || nbits == 3072 || nbits == 4096;
}

static const uint32_t kSmallPrimes[] = {
    3,   5,   7,   11,  13,  17,  19,  23,  29,  31,  37,  41,  43,  47,  53,  59,  61,  67,  71,  73,  79,  83,
    89,  97,  101, 103, 107, 109, 113, 127, 131, 137, 139, 149, 151, 157, 163, 167, 173, 179, 181, 191, 193, 197,
    199, 211, 223, 227, 229, 233, 239, 241, 251, 257, 263, 269, 271, 277, 281, 283, 293, 307, 311, 313, 317, 331,
    337, 347, 349, 353, 359, 367, 373, 379, 383, 389, 397, 401, 409, 419, 421, 431, 433, 439, 443, 449, 457, 461,
    463, 467, 479, 487, 491, 499, 503, 509, 521, 523, 541, 547, 557, 563, 569, 571, 577, 587, 593, 599, 601, 607,
    613, 617, 619, 631, 641, 643, 647, 653, 659, 661, 673, 677, 683, 691, 701, 709, 719, 727, 733, 739, 743, 751,
    757, 761, 769, 773, 787, 797, 809, 811, 821, 823, 827, 829, 839, 853, 857, 859, 863, 877, 881, 883, 887, 907,
    911, 919, 929, 937, 941, 947, 953, 967, 971, 977, 983, 991, 997};

static uint32_t mod_small(const Big& x, uint32_t d) {
  uint64_t r = 0;
  for (size_t i = x.words(); i-- > 0;) r = ((r << 32) | x.w[i]) % d;
  return (uint32_t)r;
}

// Miller-Rabin with `rounds` bases drawn from Philox (stream 0xB45E).
bool probable_prime(const Big& x, int rounds, uint64_t seed) {
  if (x.bits() < 2) return false;
  if (!x.odd()) return x.bits() == 2 && x.word(0) == 2;
  for (uint32_t sp : kSmallPrimes) {
    if (x.words() == 1 && x.w[0] == sp) return true;
    if (mod_small(x, sp) == 0) return false;
  }
  const Big one(1), xm1 = sub(x, one);
  int s = 0;
  while (!xm1.bit(s)) ++s;
  const Big d = shr(xm1, s);
  const Mont M(x);
  const Big mone = M.to(xm1), mo = M.R1;
  for (int r = 0; r < rounds; ++r) {
    // base in [2, x-2]
    Big a;
    a.w.resize(x.words());
    for (size_t j = 0; j < a.w.size(); j += 4) {
      const U4 v = philox4x32_10(U4{(uint32_t)j, (uint32_t)r, 0xB45Eu, (uint32_t)x.w[0]}, (uint32_t)seed,
                                 (uint32_t)(seed >> 32));
      const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
      for (int i = 0; i < 4 && j + i < a.w.size(); ++i) a.w[j + i] = w4[i];
    }
    a.trim();
    a = add(mod(a, sub(x, Big(3))), Big(2));
    Big y = M.to(a), acc = M.R1;
    for (int i = d.bits() - 1; i >= 0; --i) {
      acc = M.mul(acc, acc);
      if (d.bit(i)) acc = M.mul(acc, y);
    }
    if (cmp(acc, mo) == 0 || cmp(acc, mone) == 0) continue;
    bool ok = false;
    for (int i = 1; i < s; ++i) {
      acc = M.mul(acc, acc);
      if (cmp(acc, mone) == 0) { ok = true; break; }
      if (cmp(acc, mo) == 0) break;
    }
    if (!ok) return false;
  }
  return true;
}

template <int MAXS>
static bool sched_for(const Big& E, int w, Sched<MAXS>& out) {
  std::memset(&out, 0, sizeof(out));
  out.w = w;
  if (E.zero()) return false;
  int n = 0, muls = 1 + ((1 << (w - 1)) - 1);  // x^2 and the table of odd powers
  auto push = [&](int nsq, int idx) {
    while (nsq > 255) {
      if (n >= MAXS) return false;
      out.step[n++] = (uint16_t)(255 << 8);
      muls += 255;
      nsq -= 255;
    }
    if (n >= MAXS) return false;
    out.step[n++] = (uint16_t)((nsq << 8) | (idx + 1));
    muls += nsq + (idx >= 0 ? 1 : 0);
    return true;
  };
  int i = E.bits() - 1;
  bool first = true;
  int pending = 0;
  while (i >= 0) {
    if (!E.bit(i)) { ++pending; --i; continue; }
    int j = i - w + 1 < 0 ? 0 : i - w + 1;
    while (!E.bit(j)) ++j;
    uint32_t val = 0;
    for (int b = i; b >= j; --b) val = (val << 1) | (uint32_t)E.bit(b);
    const int idx = (int)(val - 1) / 2;
    if (first) {
      if (n >= MAXS) return false;
      out.step[n++] = (uint16_t)(idx + 1);  // load, no squarings
      first = false;
    } else {
      if (!push(pending + (i - j + 1), idx)) return false;
    }
    pending = 0;
    i = j - 1;
  }
  if (pending && !push(pending, -1)) return false;
  out.nsteps = n;
  out.montmuls = muls;
  return true;
}

template <int MAXS>
bool build_sched(const Big& E, int w, Sched<MAXS>& out) {
  if (w) return sched_for(E, w, out);
  bool any = false;
  Sched<MAXS> tmp;
  for (int ww = 3; ww <= kMaxWin; ++ww) {
    if (!sched_for(E, ww, tmp)) continue;
    if (!any || tmp.montmuls < out.montmuls) { out = tmp; any = true; }
  }
  return any;
}

// As build_sched, with the automatic width limited to `cap` (the window table
// of a launch is sized for one width).
template <int MAXS>
static bool build_sched_capped(const Big& E, int w, int cap, Sched<MAXS>& out) {
  if (w) return sched_for(E, w, out);
  bool any = false;
  Sched<MAXS> tmp;
  for (int ww = 3; ww <= cap; ++ww) {
    if (!sched_for(E, ww, tmp)) continue;
    if (!any || tmp.montmuls < out.montmuls) { out = tmp; any = true; }
  }
  return any;
}

template <int L>
void fill_mod(ModConst<L>& m, const Big& N) {
  std::memset(&m, 0, sizeof(m));
  const Mont M(N, L);
  N.to_words(m.n, L);
  M.R1.to_words(m.r1, L);
  M.R2.to_words(m.r2, L);
  M.R3.to_words(m.r3, L);
  m.np = M.np;
}

static Big inv_mod_prime(const Big& a, const Big& p) { return powmod(a, sub(p, Big(2)), p); }

int key_from_primes(const Big& p0, const Big& q0, pc2_key** out) {
  Big p = p0, q = q0;
  if (cmp(p, q) == 0) return PC2_EKEY;
  if (cmp(p, q) > 0) std::swap(p, q);
  const int half = p.bits();
  if (q.bits() != half || !supported_nbits(2 * half) || !p.odd() || !q.odd()) return PC2_EINVAL;
  if (!probable_prime(p, 16, 1) || !probable_prime(q, 16, 2)) return PC2_EKEY;
  const Big one(1), p1 = sub(p, one), q1 = sub(q, one);
  // gcd(n, lambda) = 1  <=>  p does not divide q-1 and q does not divide p-1
  if (mod(q1, p).zero() || mod(p1, q).zero()) return PC2_EKEY;
  std::unique_ptr<pc2_key> k(new (std::nothrow) pc2_key);
  if (!k) return PC2_ENOMEM;
  k->nbits = 2 * half;
  k->Lh = k->nbits / 32;
  k->priv = true;
  k->p = p;
  k->q = q;
  k->n = mul(p, q);
  k->n2 = mul(k->n, k->n);
  // lambda = (p-1)(q-1) / gcd(p-1, q-1)
  Big a = p1, b = q1;
  while (!b.zero()) { Big t = mod(a, b); a = b; b = t; }
  Big prod = mul(p1, q1), lam;
  {
    // exact division prod / a by binary long division
    Big r;
    lam.w.assign(prod.words(), 0);
    for (int i = prod.bits() - 1; i >= 0; --i) {
      r = shl(r, 1);
      if (prod.bit(i)) { if (r.w.empty()) r.w.push_back(1); else r.w[0] |= 1u; }
      if (cmp(r, a) >= 0) { r = sub(r, a); lam.w[(size_t)i / 32] |= 1u << (i % 32); }
    }
    lam.trim();
  }
  k->lambda = lam;
  // mu = lambda^-1 mod n = lambda^(phi(n) - 1) mod n
  k->mu = powmod(lam, sub(prod, one), k->n);
  *out = k.release();
  return PC2_OK;
}

template <int Lh>
int make_enc_crt(const pc2_key& k, int w, EncCrtParams<Lh>& P) {
  if (!k.priv) return PC2_EKEY;
  std::memset(&P, 0, sizeof(P));
  const Big p2 = mul(k.p, k.p), q2 = mul(k.q, k.q), one(1);
  fill_mod(P.mp, p2);
  fill_mod(P.mq, q2);
  const Big ep = mod(k.n, mul(k.p, sub(k.p, one))), eq = mod(k.n, mul(k.q, sub(k.q, one)));
  if (!build_sched(ep, w, P.ep) || !build_sched(eq, w, P.eq)) return PC2_EUNSUPPORTED;
  // lifted route: s = r^(h' mod (h-1)) mod h, then s^h mod h^2
  const int cap = P.ep.w > P.eq.w ? P.ep.w : P.eq.w;
  auto lift = [&](LiftConst<Lh>& C, const Big& h, const Big& ho, const Big& h2) {
    fill_mod(C.h, h);
    if (!build_sched_capped(mod(ho, sub(h, one)), w, cap, C.e1)) return false;
    if (!build_sched_capped(h, w, cap, C.e2)) return false;
    mod(shl(one, 3 * 16 * Lh), h2).to_words(C.lift, Lh);  // R_h^3, R_h = 2^(16 Lh)
    return true;
  };
  if (!lift(P.lp, k.p, k.q, p2) || !lift(P.lq, k.q, k.p, q2)) return PC2_EUNSUPPORTED;
  k.n.to_words(P.nwords, Lh);
  p2.to_words(P.p2, Lh);
  // (p^2)^-1 mod q^2 = (p^-1 mod q^2)^2, p^-1 mod q^2 = p^(q(q-1) - 1)
  const Big pinv = powmod(k.p, sub(mul(k.q, sub(k.q, one)), one), q2);
  const Big pinv2 = mulmod(pinv, pinv, q2);
  const Mont Mq(q2, Lh);
  mulmod(pinv2, Mq.R1, q2).to_words(P.pinv2R, Lh);
  P.split = ~0ull;
  return PC2_OK;
}

template <int L2>
int make_enc_pub(const pc2_key& k, int w, EncPubParams<L2>& P) {
  std::memset(&P, 0, sizeof(P));
  fill_mod(P.m, k.n2);
  if (!build_sched(k.n, w, P.e)) return PC2_EUNSUPPORTED;
  k.n.to_words(P.nwords, L2 / 2);
  return PC2_OK;
}

template <int Lh>
int make_dec(const pc2_key& k, int w, DecParams<Lh>& P) {
  if (!k.priv) return PC2_EKEY;
  constexpr int Lp = Lh / 2;
  std::memset(&P, 0, sizeof(P));
  const Big one(1), p2 = mul(k.p, k.p), q2 = mul(k.q, k.q);
  fill_mod(P.mp, p2);
  fill_mod(P.mq, q2);
  if (!build_sched(sub(k.p, one), w, P.ep) || !build_sched(sub(k.q, one), w, P.eq)) return PC2_EUNSUPPORTED;
  k.p.to_words(P.p, Lp);
  k.q.to_words(P.q, Lp);
  const Mont Mp(k.p, Lp), Mq(k.q, Lp);
  P.pnp = Mp.np;
  P.qnp = Mq.np;
  // h_p = (-q)^-1 mod p, h_q = (-p)^-1 mod q  (with g = n + 1)
  const Big hp = inv_mod_prime(sub(k.p, mod(k.q, k.p)), k.p);
  const Big hq = inv_mod_prime(sub(k.q, k.p), k.q);
  mulmod(hp, Mp.R1, k.p).to_words(P.hpR, Lp);
  mulmod(hq, Mq.R1, k.q).to_words(P.hqR, Lp);
  mulmod(inv_mod_prime(k.p, k.q), Mq.R1, k.q).to_words(P.pinvqR, Lp);
  inv_pow2(k.p, Lp).to_words(P.pinvlo, Lp);
  inv_pow2(k.q, Lp).to_words(P.qinvlo, Lp);
  return PC2_OK;
}

template <int L2>
int make_hom(const pc2_key& k, int w, int ngroups, HomParams<L2>& P) {
  std::memset(&P, 0, sizeof(P));
  fill_mod(P.m, k.n2);
  const Mont M(k.n2, L2);
  // R^k mod n^2 undoes the k-1 factors R^-1 of k-1 products and the last one
  Big rk = M.R1;
  for (int i = 1; i < ngroups; ++i) rk = mulmod(rk, M.R1, k.n2);
  rk.to_words(P.rk, L2);
  P.ngroups = ngroups;
  P.w = w ? w : 4;
  return PC2_OK;
}

#define PC2_KEY_INST_H(Lh)                                         \
  template int make_enc_crt<Lh>(const pc2_key&, int, EncCrtParams<Lh>&); \
  template int make_dec<Lh>(const pc2_key&, int, DecParams<Lh>&);
#define PC2_KEY_INST_2(L2)                                          \
  template int make_enc_pub<L2>(const pc2_key&, int, EncPubParams<L2>&); \
  template int make_hom<L2>(const pc2_key&, int, int, HomParams<L2>&);
PC2_KEY_INST_H(8)
PC2_KEY_INST_H(16)
PC2_KEY_INST_H(32)
PC2_KEY_INST_H(64)
PC2_KEY_INST_H(96)
PC2_KEY_INST_H(128)
PC2_KEY_INST_2(16)
PC2_KEY_INST_2(32)
PC2_KEY_INST_2(64)
PC2_KEY_INST_2(128)
PC2_KEY_INST_2(192)
PC2_KEY_INST_2(256)

}  // namespace pc2
