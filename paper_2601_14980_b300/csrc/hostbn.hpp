// hostbn.hpp -- host-side multi-precision integers for key set-up in libpc2.
//
// Off the hot path: used once per key to generate primes and to derive the
// Montgomery constants, CRT constants and exponent schedules that the
// kernels receive.  Little-endian vectors of 32-bit words, always trimmed.
#pragma once
#include <algorithm>
#include <cstdint>
#include <stdexcept>
#include <vector>

namespace pc2 {

struct Big {
  std::vector<uint32_t> w;  // little-endian, no leading zero words

  Big() = default;
  explicit Big(uint64_t v) {
    if (v) w.push_back((uint32_t)v);
    if (v >> 32) w.push_back((uint32_t)(v >> 32));
  }
  static Big from_words(const uint32_t* p, size_t n) {
    Big b;
    b.w.assign(p, p + n);
    b.trim();
    return b;
  }
  void trim() { while (!w.empty() && w.back() == 0) w.pop_back(); }
  bool zero() const { return w.empty(); }
  size_t words() const { return w.size(); }
  uint32_t word(size_t i) const { return i < w.size() ? w[i] : 0u; }
  int bits() const {
    if (w.empty()) return 0;
    int b = 32 * (int)(w.size() - 1);
    uint32_t t = w.back();
    while (t) { ++b; t >>= 1; }
    return b;
  }
  int bit(int i) const { return (word((size_t)i / 32) >> (i % 32)) & 1; }
  bool odd() const { return !w.empty() && (w[0] & 1u); }
  void to_words(uint32_t* out, size_t n) const {
    if (w.size() > n) throw std::runtime_error("Big::to_words: value too wide");
    for (size_t i = 0; i < n; ++i) out[i] = word(i);
  }
};

inline int cmp(const Big& a, const Big& b) {
  if (a.w.size() != b.w.size()) return a.w.size() < b.w.size() ? -1 : 1;
  for (size_t i = a.w.size(); i-- > 0;)
    if (a.w[i] != b.w[i]) return a.w[i] < b.w[i] ? -1 : 1;
  return 0;
}

inline Big add(const Big& a, const Big& b) {
  Big r;
  size_t n = std::max(a.words(), b.words());
  r.w.resize(n + 1);
  uint64_t c = 0;
  for (size_t i = 0; i < n; ++i) {
    c += (uint64_t)a.word(i) + b.word(i);
    r.w[i] = (uint32_t)c;
    c >>= 32;
  }
  r.w[n] = (uint32_t)c;
  r.trim();
  return r;
}

inline Big sub(const Big& a, const Big& b) {  // a >= b
  if (cmp(a, b) < 0) throw std::runtime_error("Big::sub underflow");
  Big r;
  r.w.resize(a.words());
  int64_t br = 0;
  for (size_t i = 0; i < a.words(); ++i) {
    int64_t d = (int64_t)a.w[i] - b.word(i) - br;
    br = d < 0;
    r.w[i] = (uint32_t)(d + (br << 32));
  }
  r.trim();
  return r;
}

inline Big mul(const Big& a, const Big& b) {
  Big r;
  if (a.zero() || b.zero()) return r;
  r.w.assign(a.words() + b.words(), 0);
  for (size_t i = 0; i < a.words(); ++i) {
    uint64_t c = 0;
    for (size_t j = 0; j < b.words(); ++j) {
      c += (uint64_t)a.w[i] * b.w[j] + r.w[i + j];
      r.w[i + j] = (uint32_t)c;
      c >>= 32;
    }
    r.w[i + b.words()] = (uint32_t)c;
  }
  r.trim();
  return r;
}

inline Big shl(const Big& a, int s) {
  if (a.zero()) return a;
  Big r;
  int ws = s / 32, bs = s % 32;
  r.w.assign(a.words() + ws + 1, 0);
  for (size_t i = 0; i < a.words(); ++i) {
    r.w[i + ws] |= a.w[i] << bs;
    if (bs) r.w[i + ws + 1] |= a.w[i] >> (32 - bs);
  }
  r.trim();
  return r;
}

inline Big shr(const Big& a, int s) {
  Big r;
  int ws = s / 32, bs = s % 32;
  if ((size_t)ws >= a.words()) return r;
  r.w.assign(a.words() - ws, 0);
  for (size_t i = 0; i < r.words(); ++i) {
    r.w[i] = a.w[i + ws] >> bs;
    if (bs && i + ws + 1 < a.words()) r.w[i] |= a.w[i + ws + 1] << (32 - bs);
  }
  r.trim();
  return r;
}

// Remainder by binary long division: one bit of the dividend per step.
inline Big mod(const Big& a, const Big& m) {
  if (m.zero()) throw std::runtime_error("Big::mod by zero");
  if (cmp(a, m) < 0) return a;
  Big r;
  for (int i = a.bits() - 1; i >= 0; --i) {
    r = shl(r, 1);
    if (a.bit(i)) {
      if (r.w.empty()) r.w.push_back(1); else r.w[0] |= 1u;
    }
    if (cmp(r, m) >= 0) r = sub(r, m);
  }
  return r;
}

inline Big mulmod(const Big& a, const Big& b, const Big& m) { return mod(mul(a, b), m); }

// x^{-1} mod 2^32 for odd x (Newton: each step doubles the correct bits).
inline uint32_t inv32(uint32_t x) {
  uint32_t y = x;  // correct to 3 bits for odd x
  for (int i = 0; i < 5; ++i) y *= 2u - x * y;
  return y;
}

// Low k words of a (a mod 2^(32k)).
inline Big low_words(const Big& a, int k) {
  Big r;
  r.w.assign(a.w.begin(), a.w.begin() + std::min<size_t>(a.words(), (size_t)k));
  r.trim();
  return r;
}

// x^{-1} mod 2^(32k) for odd x, by Newton iteration y <- y (2 - x y).
inline Big inv_pow2(const Big& x, int k) {
  Big y(inv32(x.word(0)));
  Big two_k = shl(Big(1), 32 * k);
  for (int bits = 32; bits < 32 * k; bits *= 2) {
    Big xy = low_words(mul(x, y), k);
    Big t = low_words(sub(add(Big(2), two_k), xy), k);  // 2 - xy mod 2^(32k)
    y = low_words(mul(y, t), k);
  }
  return y;
}

// Montgomery arithmetic mod an odd N of L words (R = 2^(32L)).
struct Mont {
  Big N;
  int L = 0;
  uint32_t np = 0;  // -N^{-1} mod 2^32
  Big R1, R2, R3;   // R, R^2, R^3 mod N

  explicit Mont(const Big& n, int limbs = 0) : N(n) {
    if (!n.odd()) throw std::runtime_error("Mont: even modulus");
    L = limbs ? limbs : (int)n.words();
    if ((int)n.words() > L) throw std::runtime_error("Mont: modulus wider than limbs");
    np = 0u - inv32(n.w[0]);
    R1 = mod(shl(Big(1), 32 * L), N);
    R2 = mulmod(R1, R1, N);
    R3 = mulmod(R2, R1, N);
  }
  // a * b / R mod N for a, b < N (CIOS with 64-bit host words).
  Big mul(const Big& a, const Big& b) const {
    std::vector<uint32_t> t(L + 2, 0);
    for (int i = 0; i < L; ++i) {
      uint64_t c = 0;
      const uint64_t bi = b.word(i);
      for (int j = 0; j < L; ++j) {
        c += (uint64_t)t[j] + a.word(j) * bi;
        t[j] = (uint32_t)c;
        c >>= 32;
      }
      c += t[L];
      t[L] = (uint32_t)c;
      t[L + 1] = (uint32_t)(c >> 32);
      const uint64_t m = (uint32_t)(t[0] * np);
      c = ((uint64_t)t[0] + m * N.word(0)) >> 32;
      for (int j = 1; j < L; ++j) {
        c += (uint64_t)t[j] + m * N.word(j);
        t[j - 1] = (uint32_t)c;
        c >>= 32;
      }
      c += t[L];
      t[L - 1] = (uint32_t)c;
      t[L] = t[L + 1] + (uint32_t)(c >> 32);
    }
    Big r = Big::from_words(t.data(), L + 1);
    if (cmp(r, N) >= 0) r = sub(r, N);
    return r;
  }
  Big to(const Big& a) const { return mul(mod(a, N), R2); }
  Big from(const Big& a) const { return mul(a, Big(1)); }
  Big pow(const Big& base, const Big& e) const {
    Big x = to(base), acc = R1;
    for (int i = e.bits() - 1; i >= 0; --i) {
      acc = mul(acc, acc);
      if (e.bit(i)) acc = mul(acc, x);
    }
    return from(acc);
  }
};

inline Big powmod(const Big& b, const Big& e, const Big& m) { return Mont(m).pow(b, e); }

}  // namespace pc2
