// mont.cuh -- device big-integer core of libpc2 (sm_103a).
//
// Numbers are little-endian 32-bit limbs.  An element (one ciphertext or
// plaintext being processed) is owned by a GROUP of T consecutive lanes of a
// warp; lane k of the group holds limbs [k*S, (k+1)*S) of the L = S*T limb
// operands in registers.  T divides 32, so a group never spans warps and only
// __syncwarp() is ever needed.
//
// mont_mul  -- Montgomery product a*b/R mod N by coarsely integrated operand
//              scanning (CIOS, Koc/Acar/Kaliski 1996): one row t += a*b_i
//              (per word one 32x32->64 product and a 64-bit add, the carry
//              in a register, two rows per loop trip; at 128 limbs two
//              carry-flag chains, low then high halves), one row t += m*N
//              with m = t_0 * (-N^-1) mod 2^32, then a one-word shift.  Each lane keeps the carry word of its
//              segment separately (a redundant representation); the shift
//              hands every lane the low word of its upper neighbour by a
//              warp shuffle, and carries are resolved once, after the last
//              row.  b is read one word per row from shared memory.
// modexp_sched -- left-to-right sliding-window exponentiation with a fixed,
//              warp-uniform schedule (every lane runs the same squarings and
//              multiplies; only the data differ).
// modexp_var -- fixed-window exponentiation by a per-element 64-bit exponent,
//              uniform control flow (digit 0 multiplies by the Montgomery 1).
//
// Glue (g_*) -- word-serial helpers for the few steps per element outside the
// exponentiation (conversions, CRT recombination, exact division).  They run
// on global-memory scratch columns; with T > 1 all lanes of a group execute
// them redundantly on the same data (one instruction stream under SIMT).
#pragma once
#include <cstdint>
#include "pc2_params.h"

namespace pc2 {

#define PC2_FULL 0xffffffffu

// ---------------------------------------------------------------- PTX carry chains
__device__ __forceinline__ void mad_lo_cc(uint32_t& t, uint32_t a, uint32_t b) {
  asm volatile("mad.lo.cc.u32 %0, %1, %2, %0;" : "+r"(t) : "r"(a), "r"(b));
}
__device__ __forceinline__ void madc_lo_cc(uint32_t& t, uint32_t a, uint32_t b) {
  asm volatile("madc.lo.cc.u32 %0, %1, %2, %0;" : "+r"(t) : "r"(a), "r"(b));
}
__device__ __forceinline__ void mad_hi_cc(uint32_t& t, uint32_t a, uint32_t b) {
  asm volatile("mad.hi.cc.u32 %0, %1, %2, %0;" : "+r"(t) : "r"(a), "r"(b));
}
__device__ __forceinline__ void madc_hi_cc(uint32_t& t, uint32_t a, uint32_t b) {
  asm volatile("madc.hi.cc.u32 %0, %1, %2, %0;" : "+r"(t) : "r"(a), "r"(b));
}
__device__ __forceinline__ void addc_cc_z(uint32_t& t) { asm volatile("addc.cc.u32 %0, %0, 0;" : "+r"(t)); }
__device__ __forceinline__ void addc_z(uint32_t& t) { asm volatile("addc.u32 %0, %0, 0;" : "+r"(t)); }

// ---------------------------------------------------------------- lane groups
template <int T>
struct Grp {
  int k;     // lane index inside the group
  int base;  // warp lane of the group's lane 0
  __device__ Grp() : k((int)(threadIdx.x & (T - 1))), base((int)(threadIdx.x & 31u) & ~(T - 1)) {}
  __device__ __forceinline__ uint32_t bcast(uint32_t v, int src) const {
    if constexpr (T == 1) return v;
    else return __shfl_sync(PC2_FULL, v, src, T);
  }
  __device__ __forceinline__ uint32_t from_next(uint32_t v) const {
    if constexpr (T == 1) return 0u;
    else {
      const uint32_t x = __shfl_down_sync(PC2_FULL, v, 1, T);
      return k == T - 1 ? 0u : x;
    }
  }
  __device__ __forceinline__ uint32_t from_prev(uint32_t v) const {
    if constexpr (T == 1) return 0u;
    else {
      const uint32_t x = __shfl_up_sync(PC2_FULL, v, 1, T);
      return k == 0 ? 0u : x;
    }
  }
};

// Modulus words: from the kernel parameter block (T == 1: every lane needs all
// words and the offsets are compile-time constants) or from registers (T > 1:
// lane k needs its own segment).
struct ParamN {
  const uint32_t* n;
  __device__ __forceinline__ uint32_t operator[](int j) const { return n[j]; }
};
template <int S>
struct RegN {
  uint32_t v[S];
  __device__ __forceinline__ uint32_t operator[](int j) const { return v[j]; }
};
template <int S, int T>
__device__ __forceinline__ RegN<S> reg_n(const uint32_t* n, const Grp<T>& g) {
  RegN<S> r;
#pragma unroll
  for (int j = 0; j < S; ++j) r.v[j] = n[g.k * S + j];
  return r;
}

template <int S>
struct RegA {
  const uint32_t (&v)[S];
  __device__ __forceinline__ uint32_t operator[](int j) const { return v[j]; }
};

// Row form per operand size, as measured on B300 (every kernel family at
// its benchmark configuration, both forms bit-identical): wide products win
// at 32, 64, 96 and 256 limbs (3072-bit encryption 25 % faster, the small
// LASSO's rounds 14 %), carry-flag chains at 128 limbs (the n^2 powers and
// products of 2048-bit keys: 22 % faster).
template <int S, int T>
constexpr bool wide_rows() {
  return S * T != 128;
}

// Carry-flag form: the low halves of the 32x32 products (mad.lo.cc /
// madc.lo.cc), then the high halves.
template <int S, class A>
__device__ __forceinline__ void row_mac_cc(uint32_t (&t)[S], uint32_t& c0, uint32_t& c1, const A& a, uint32_t b) {
  mad_lo_cc(t[0], a[0], b);
#pragma unroll
  for (int j = 1; j < S; ++j) madc_lo_cc(t[j], a[j], b);
  addc_cc_z(c0);
  addc_z(c1);
  mad_hi_cc(t[1], a[0], b);
#pragma unroll
  for (int j = 1; j < S - 1; ++j) madc_hi_cc(t[j + 1], a[j], b);
  madc_hi_cc(c0, a[S - 1], b);
  addc_z(c1);
}

// t[0..S-1], (c0, c1) += a[0..S-1] * b   (c0, c1: carry words above the segment)
template <int S, class A>
__device__ __forceinline__ void row_mac(uint32_t (&t)[S], uint32_t& c0, uint32_t& c1, const A& a, uint32_t b) {
  static_assert(S >= 2, "segments of at least two limbs");
  // each step a_j b + t_j + c < 2^64: one wide product and a 64-bit add,
  // the carry in a register (no carry-flag chain)
  uint32_t c = 0u;
#pragma unroll
  for (int j = 0; j < S; ++j) {
    const uint64_t p = (uint64_t)a[j] * b + t[j] + c;
    t[j] = (uint32_t)p;
    c = (uint32_t)(p >> 32);
  }
  const uint64_t v = (uint64_t)c0 + c;
  c0 = (uint32_t)v;
  c1 += (uint32_t)(v >> 32);
}

// Final step of mont_mul: t (this lane's words) plus the carry
// word (c0, c1) above the segment is < 2N; write t - N or t into a.
template <int S, int T, class NS>
__device__ __forceinline__ void mont_finish(uint32_t (&a)[S], uint32_t (&t)[S], uint32_t c0, uint32_t c1, const NS& n,
                                            const Grp<T>& g) {
  if constexpr (T == 1) {
    // t + c0 R < 2N: subtract N when c0 != 0 or t >= N.
    uint32_t br;
    asm volatile("sub.cc.u32 %0, %1, %2;" : "=r"(a[0]) : "r"(t[0]), "r"(n[0]));
#pragma unroll
    for (int j = 1; j < S; ++j) asm volatile("subc.cc.u32 %0, %1, %2;" : "=r"(a[j]) : "r"(t[j]), "r"(n[j]));
    asm volatile("subc.u32 %0, 0, 0;" : "=r"(br));
    const bool keep = (c0 == 0u) && (br != 0u);
#pragma unroll
    for (int j = 0; j < S; ++j) a[j] = keep ? t[j] : a[j];
  } else {
    // Resolve the per-lane carry words: T-1 ripple steps.
#pragma unroll
    for (int it = 0; it < T - 1; ++it) {
      const uint32_t i0 = g.from_prev(c0), i1 = g.from_prev(c1);
      if (g.k != T - 1) { c0 = 0u; c1 = 0u; }
      asm volatile("add.cc.u32 %0, %0, %1;" : "+r"(t[0]) : "r"(i0));
      asm volatile("addc.cc.u32 %0, %0, %1;" : "+r"(t[1]) : "r"(i1));
#pragma unroll
      for (int j = 2; j < S; ++j) addc_cc_z(t[j]);
      addc_cc_z(c0);
      addc_z(c1);
    }
    const uint32_t top = g.bcast(c0, T - 1);
    // Segment difference d = t - n (borrow-in 0), its borrow-out and equality.
    uint32_t br;
    asm volatile("sub.cc.u32 %0, %1, %2;" : "=r"(a[0]) : "r"(t[0]), "r"(n[0]));
#pragma unroll
    for (int j = 1; j < S; ++j) asm volatile("subc.cc.u32 %0, %1, %2;" : "=r"(a[j]) : "r"(t[j]), "r"(n[j]));
    asm volatile("subc.u32 %0, 0, 0;" : "=r"(br));
    uint32_t nz = 0u;
#pragma unroll
    for (int j = 0; j < S; ++j) nz |= a[j];
    // Borrow look-ahead across the group: borrow into lane kk+1 is
    // generate_kk | (equal_kk & borrow into kk).
    const uint32_t gb = __ballot_sync(PC2_FULL, br != 0u) >> g.base;
    const uint32_t eb = __ballot_sync(PC2_FULL, (br == 0u) && (nz == 0u)) >> g.base;
    uint32_t bin = 0u, b = 0u;
#pragma unroll
    for (int kk = 0; kk < T; ++kk) {
      if (kk == g.k) bin = b;
      b = ((gb >> kk) & 1u) | (((eb >> kk) & 1u) & b);
    }
    const bool sub = (top != 0u) || (b == 0u);
    // d - bin gives this lane's words of t - N.
    asm volatile("sub.cc.u32 %0, %0, %1;" : "+r"(a[0]) : "r"(bin));
#pragma unroll
    for (int j = 1; j < S; ++j) asm volatile("subc.cc.u32 %0, %0, 0;" : "+r"(a[j]));
#pragma unroll
    for (int j = 0; j < S; ++j) a[j] = sub ? a[j] : t[j];
  }
}

// a <- a * b / R mod N.  a: this lane's segment (registers, a < R);
// b: the group's operand in shared memory, word i at bcol[i * bstride] (b < N).
template <int S, int T, class NS>
__device__ __forceinline__ void mont_mul(uint32_t (&a)[S], const uint32_t* __restrict__ bcol, int bstride, const NS& n,
                                         uint32_t np, const Grp<T>& g) {
  constexpr int L = S * T;
  uint32_t t[S];
#pragma unroll
  for (int j = 0; j < S; ++j) t[j] = 0u;
  uint32_t c0 = 0u, c1 = 0u;
  const RegA<S> av{a};
  auto step = [&](int i) {
    const uint32_t b = bcol[i * bstride];
    if constexpr (wide_rows<S, T>()) row_mac<S>(t, c0, c1, av, b);
    else row_mac_cc<S>(t, c0, c1, av, b);
    const uint32_t m = g.bcast(t[0] * np, 0);
    if constexpr (wide_rows<S, T>()) row_mac<S>(t, c0, c1, n, m);
    else row_mac_cc<S>(t, c0, c1, n, m);
    const uint32_t up = g.from_next(t[0]);
#pragma unroll
    for (int j = 0; j < S - 1; ++j) t[j] = t[j + 1];
    asm volatile("add.cc.u32 %0, %1, %2;" : "=r"(t[S - 1]) : "r"(up), "r"(c0));
    asm volatile("addc.u32 %0, %1, 0;" : "=r"(c0) : "r"(c1));
    c1 = 0u;
  };
  if constexpr (wide_rows<S, T>()) {
#pragma unroll 2
    for (int i = 0; i < L; ++i) step(i);
  } else {
#pragma unroll 1
    for (int i = 0; i < L; ++i) step(i);
  }
  mont_finish<S, T>(a, t, c0, c1, n, g);
}

// ---------------------------------------------------------------- columns
// Word j of a per-group array: p[j * s] (interleaved so a warp's accesses coalesce).
struct Col {
  uint32_t* p;
  int s;
  __device__ __forceinline__ uint32_t& operator[](int j) const { return p[(size_t)j * s]; }
  __device__ __forceinline__ Col off(int j) const { return Col{p + (size_t)j * s, s}; }
};

template <int S, int T>
__device__ __forceinline__ void load_seg(uint32_t (&a)[S], const Col& c, const Grp<T>& g) {
#pragma unroll
  for (int j = 0; j < S; ++j) a[j] = c[g.k * S + j];
}
template <int S, int T>
__device__ __forceinline__ void store_seg(const Col& c, const uint32_t (&a)[S], const Grp<T>& g) {
#pragma unroll
  for (int j = 0; j < S; ++j) c[g.k * S + j] = a[j];
}

// ---------------------------------------------------------------- exponentiation
// a <- a^E (Montgomery domain).  tab: scratch column for the 2^(w-1) odd powers
// (entry e at words [e*L, (e+1)*L)); bsh: the group's shared operand column.
// One call site of mont_mul: a uniform state machine picks what goes into the
// two operands before each product (x^2, the table of odd powers, then the
// schedule's squarings and table multiplies).
template <int S, int T, int MAXS, class NS>
__device__ __forceinline__ void modexp_sched(uint32_t (&a)[S], const Sched<MAXS>& E, const Col tab, const Col bsh,
                                             const NS& n, uint32_t np, const Grp<T>& g) {
  constexpr int L = S * T;
  const int ntab = 1 << (E.w - 1);
  const int idx0 = (int)(E.step[0] & 0xffu) - 1;
  int phase = 0, e = 1, s = 1, q = 0;
  store_seg(tab, a, g);
  store_seg(bsh, a, g);
  __syncwarp();
  for (;;) {
    mont_mul<S, T>(a, bsh.p, bsh.s, n, np, g);
    __syncwarp();
    if (phase == 0) {  // a = x^2: keep it as the fixed multiplier of the table
      store_seg(bsh, a, g);
      __syncwarp();
      load_seg(a, tab, g);
      phase = 1;
      if (ntab > 1) continue;
      phase = 2;
      load_seg(a, tab.off(idx0 * L), g);
    } else if (phase == 1) {  // a = x^(2e+1)
      store_seg(tab.off(e * L), a, g);
      if (++e < ntab) continue;
      phase = 2;
      load_seg(a, tab.off(idx0 * L), g);
    }
    bool more = false;
    while (s < E.nsteps) {
      const uint32_t st = E.step[s];
      const int nsq = (int)(st >> 8), idx = (int)(st & 0xffu) - 1;
      if (q < nsq) {  // square
        ++q;
        store_seg(bsh, a, g);
        __syncwarp();
        more = true;
        break;
      }
      if (q == nsq && idx >= 0) {  // multiply by the table entry
        ++q;
        store_seg(bsh, a, g);
        __syncwarp();
        load_seg(a, tab.off(idx * L), g);
        more = true;
        break;
      }
      ++s;
      q = 0;
    }
    if (!more) break;
  }
}

// a <- a^k (Montgomery domain) for a per-element exponent given as nd digits
// of w bits, most significant first: digit(pos) returns digit pos (pos = nd-1
// down to 0).  tab: 2^w entries (tab[d] = x^d, tab[0] = R mod N); nd is
// warp-uniform.  Every digit costs w squarings and one multiply, so control
// flow is the same for every lane.
template <int S, int T, class NS, class DigitFn>
__device__ __forceinline__ void modexp_digits(uint32_t (&a)[S], DigitFn digit, int w, int nd, const uint32_t* r1,
                                              const Col tab, const Col bsh, const NS& n, uint32_t np,
                                              const Grp<T>& g) {
  constexpr int L = S * T;
  const int ntab = 1 << w;
  // tab[0] = 1 (Montgomery), tab[1] = x, tab[d] = tab[d-1] * x
#pragma unroll
  for (int j = 0; j < S; ++j) tab[g.k * S + j] = r1[g.k * S + j];
  store_seg(tab.off(L), a, g);
  store_seg(bsh, a, g);
  __syncwarp();
  int phase = (ntab > 2) ? 1 : 2, d = 2, pos = nd - 1, sq = 0;
  if (phase == 2) {
    // no table products needed: start the digit loop directly
    load_seg(a, tab.off(digit(pos) * L), g);
    --pos;
    if (pos < 0) return;
    store_seg(bsh, a, g);
    __syncwarp();
    sq = 1;
  }
  for (;;) {
    mont_mul<S, T>(a, bsh.p, bsh.s, n, np, g);
    __syncwarp();
    if (phase == 1) {
      store_seg(tab.off(d * L), a, g);
      if (++d < ntab) continue;
      phase = 2;
      load_seg(a, tab.off(digit(pos) * L), g);
      --pos;
      if (pos < 0) return;
      store_seg(bsh, a, g);
      __syncwarp();
      sq = 1;
      continue;
    }
    // phase 2: sq in 1..w = squarings done for the current digit; w+1 = multiply done
    if (sq < w) {
      ++sq;
      store_seg(bsh, a, g);
      __syncwarp();
      continue;
    }
    if (sq == w) {
      ++sq;
      store_seg(bsh, a, g);
      __syncwarp();
      load_seg(a, tab.off(digit(pos) * L), g);
      continue;
    }
    // multiply done: next digit
    --pos;
    if (pos < 0) return;
    sq = 1;
    store_seg(bsh, a, g);
    __syncwarp();
  }
}

// a <- a^k (Montgomery domain) for a per-element exponent k < 2^64 with
// fixed windows of w bits over nd digits (warp-uniform).
template <int S, int T, class NS>
__device__ __forceinline__ void modexp_var(uint32_t (&a)[S], uint64_t k, int w, int nd, const uint32_t* r1,
                                           const Col tab, const Col bsh, const NS& n, uint32_t np, const Grp<T>& g) {
  const uint64_t mask = ((uint64_t)1 << w) - 1u;
  modexp_digits<S, T>(a, [&](int pos) { return (int)((k >> (pos * w)) & mask); }, w, nd, r1, tab, bsh, n, np, g);
}

// ---------------------------------------------------------------- glue (word-serial)
struct PArr {
  const uint32_t* p;
  __device__ __forceinline__ uint32_t operator[](int j) const { return p[j]; }
};
__device__ __forceinline__ void g_zero(const Col& d, int len) {
  for (int j = 0; j < len; ++j) d[j] = 0u;
}
__device__ __forceinline__ void g_copy(const Col& d, const Col& s, int len) {
  for (int j = 0; j < len; ++j) d[j] = s[j];
}
__device__ __forceinline__ void g_copy_param(const Col& d, const uint32_t* s, int len) {
  for (int j = 0; j < len; ++j) d[j] = s[j];
}
// a >= b (len words)
template <class B>
__device__ __forceinline__ bool g_ge(const Col& a, const B& b, int len) {
  for (int j = len - 1; j >= 0; --j) {
    const uint32_t x = a[j], y = b[j];
    if (x != y) return x > y;
  }
  return true;
}
// d = a - b, returns the borrow (len words)
template <class B>
__device__ __forceinline__ uint32_t g_sub(const Col& d, const Col& a, const B& b, int len) {
  uint64_t br = 0;
  for (int j = 0; j < len; ++j) {
    const uint64_t x = a[j], y = (uint64_t)b[j] + br;
    d[j] = (uint32_t)(x - y);
    br = x < y;
  }
  return (uint32_t)br;
}
// d = a + b, returns the carry (len words)
template <class B>
__device__ __forceinline__ uint32_t g_add(const Col& d, const Col& a, const B& b, int len) {
  uint64_t c = 0;
  for (int j = 0; j < len; ++j) {
    c += (uint64_t)a[j] + b[j];
    d[j] = (uint32_t)c;
    c >>= 32;
  }
  return (uint32_t)c;
}
// d = (a + b) mod N for a, b < N
__device__ __forceinline__ void g_addmod(const Col& d, const Col& a, const Col& b, const uint32_t* N, int len) {
  const uint32_t c = g_add(d, a, b, len);
  if (c || g_ge(d, PArr{N}, len)) g_sub(d, d, PArr{N}, len);
}
// Word-serial CIOS: d = a * b / R mod N, R = 2^(32 len); a < R, b < N.
// t: temporary column of len + 2 words.  d may alias a or b.
__device__ __forceinline__ void g_mont(const Col d, const Col a, const Col b, const uint32_t* N, uint32_t np, int len,
                                    const Col t) {
  for (int j = 0; j < len + 2; ++j) t[j] = 0u;
  for (int i = 0; i < len; ++i) {
    const uint64_t bi = b[i];
    uint64_t c = 0;
    for (int j = 0; j < len; ++j) {
      c += (uint64_t)t[j] + (uint64_t)a[j] * bi;
      t[j] = (uint32_t)c;
      c >>= 32;
    }
    c += t[len];
    t[len] = (uint32_t)c;
    t[len + 1] = (uint32_t)(c >> 32);
    const uint64_t m = (uint32_t)(t[0] * np);
    c = ((uint64_t)t[0] + m * N[0]) >> 32;
    for (int j = 1; j < len; ++j) {
      c += (uint64_t)t[j] + m * N[j];
      t[j - 1] = (uint32_t)c;
      c >>= 32;
    }
    c += t[len];
    t[len - 1] = (uint32_t)c;
    t[len] = t[len + 1] + (uint32_t)(c >> 32);
  }
  if (t[len] || g_ge(t, PArr{N}, len)) g_sub(d, t, PArr{N}, len);
  else g_copy(d, t, len);
}
// d = Montgomery form of x mod N, x of 2*len words: mont(x_lo, R^2) + mont(x_hi, R^3).
__device__ __forceinline__ void g_to_mont_2l(const Col d, const Col x, const uint32_t* N, const uint32_t* r2,
                                            const uint32_t* r3, uint32_t np, int len, const Col t1, const Col t2,
                                            const Col tt) {
  g_copy_param(t2, r2, len);
  g_mont(t1, x, t2, N, np, len, tt);            // x_lo * R
  g_copy_param(t2, r3, len);
  g_mont(t2, x.off(len), t2, N, np, len, tt);   // x_hi * R^2 = x_hi * 2^(32 len) * R
  g_addmod(d, t1, t2, N, len);
}
// ---------------------------------------------------------------- glue products by the lane group
// The glue runs the same word-serial code on every lane of an element's
// group; its Montgomery products instead go through mont_mul: lane k holds
// words k S .. k S + S - 1 of a (S = L / T) in registers, b is read word by
// word from its column (global scratch, shared memory or a constant array,
// stride b.s), N from the pointer (T = 1) or as register segments (T > 1).
// The result is the same canonical integer as g_mont's.  d may alias a or b
// (every lane has read both before any lane writes d).  With fewer than two
// words per lane, or more than MaxS (the segment and its carries would not
// fit the kernel's register budget), it falls back to g_mont.
template <int L, int T, int MaxS = 64>
__device__ __forceinline__ void grp_mont(const Col& d, const Col& a, const Col& b, const uint32_t* N, uint32_t np,
                                         const Col& tt, const Grp<T>& g) {
  constexpr int S = L / T;
  if constexpr (S < 2 || S > MaxS) {
    g_mont(d, a, b, N, np, L, tt);
  } else {
    if constexpr (T > 1) __syncwarp();
    uint32_t x[S];
    load_seg(x, a, g);
    if constexpr (T == 1) {
      mont_mul<S, 1>(x, b.p, b.s, ParamN{N}, np, g);
    } else {
      const RegN<S> rn = reg_n<S, T>(N, g);
      mont_mul<S, T>(x, b.p, b.s, rn, np, g);
      __syncwarp();
    }
    store_seg(d, x, g);
    if constexpr (T > 1) __syncwarp();
  }
}
// A constant array (parameter block or device memory) as a column.
__device__ __forceinline__ Col const_col(const uint32_t* v) { return Col{const_cast<uint32_t*>(v), 1}; }
// g_to_mont_2l with the two products by the lane group.
template <int L, int T, int MaxS = 64>
__device__ __forceinline__ void grp_to_mont_2l(const Col& d, const Col& x, const uint32_t* N, const uint32_t* r2,
                                               const uint32_t* r3, uint32_t np, const Col& t1, const Col& t2,
                                               const Col& tt, const Grp<T>& g) {
  grp_mont<L, T, MaxS>(t1, x, const_col(r2), N, np, tt, g);         // x_lo * R
  grp_mont<L, T, MaxS>(t2, x.off(L), const_col(r3), N, np, tt, g);  // x_hi * R^2
  g_addmod(d, t1, t2, N, L);
}

// d[0..la+lb) = a[0..la) * b[0..lb) (schoolbook)
template <class B>
__device__ __forceinline__ void g_mul(const Col& d, const Col& a, int la, const B& b, int lb) {
  for (int j = 0; j < la + lb; ++j) d[j] = 0u;
  for (int i = 0; i < la; ++i) {
    const uint64_t ai = a[i];
    uint64_t c = 0;
    for (int j = 0; j < lb; ++j) {
      c += (uint64_t)d[i + j] + ai * b[j];
      d[i + j] = (uint32_t)c;
      c >>= 32;
    }
    d[i + lb] = (uint32_t)c;
  }
}
// d[0..len) = low len words of a * b (both len words)
template <class B>
__device__ __forceinline__ void g_mul_lo(const Col& d, const Col& a, const B& b, int len) {
  for (int j = 0; j < len; ++j) d[j] = 0u;
  for (int i = 0; i < len; ++i) {
    const uint64_t ai = a[i];
    uint64_t c = 0;
    for (int j = 0; j + i < len; ++j) {
      c += (uint64_t)d[i + j] + ai * b[j];
      d[i + j] = (uint32_t)c;
      c >>= 32;
    }
  }
}

// ---------------------------------------------------------------- interleaved layout
// Word j of element e in a tiled buffer of Lc-limb elements: tiles of 32
// elements, each tile stored as Lc/4 slabs of 32 x uint4 (element-major
// inside a slab), so a warp moves 512 contiguous bytes per 16-byte access.
__host__ __device__ __forceinline__ size_t tiled_index(size_t e, int j, int Lc) {
  return (((e >> 5) * (size_t)(Lc >> 2) + (size_t)(j >> 2)) << 7) + ((e & 31u) << 2) + (size_t)(j & 3);
}

}  // namespace pc2
