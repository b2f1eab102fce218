/*
 * bn.c -- plain multi-precision arithmetic for the CPU oracle (test
 * infrastructure only; see bn.h).  Every routine is the schoolbook method;
 * speed is not a goal.
 */
#include "bn.h"
#include <string.h>

static void bn_trim(bn* a) {
  while (a->len > 0 && a->w[a->len - 1] == 0) a->len--;
}

void bn_zero(bn* a) { a->len = 0; }

void bn_set_u64(bn* a, uint64_t v) {
  a->w[0] = (uint32_t)v;
  a->w[1] = (uint32_t)(v >> 32);
  a->len = 2;
  bn_trim(a);
}

void bn_from_words(bn* a, const uint32_t* w, int n) {
  for (int i = 0; i < n; i++) a->w[i] = w[i];
  a->len = n;
  bn_trim(a);
}

void bn_to_words(const bn* a, uint32_t* w, int n) {
  for (int i = 0; i < n; i++) w[i] = i < a->len ? a->w[i] : 0u;
}

void bn_copy(bn* dst, const bn* src) {
  if (dst == src) return;
  dst->len = src->len;
  for (int i = 0; i < src->len; i++) dst->w[i] = src->w[i];
}

int bn_is_zero(const bn* a) { return a->len == 0; }

int bn_cmp(const bn* a, const bn* b) {
  if (a->len != b->len) return a->len < b->len ? -1 : 1;
  for (int i = a->len - 1; i >= 0; i--)
    if (a->w[i] != b->w[i]) return a->w[i] < b->w[i] ? -1 : 1;
  return 0;
}

int bn_bitlen(const bn* a) {
  if (a->len == 0) return 0;
  uint32_t top = a->w[a->len - 1];
  int b = 0;
  while (top) { b++; top >>= 1; }
  return 32 * (a->len - 1) + b;
}

int bn_bit(const bn* a, int i) {
  int wi = i / 32;
  if (wi >= a->len) return 0;
  return (a->w[wi] >> (i % 32)) & 1u;
}

void bn_add(bn* r, const bn* a, const bn* b) {
  int n = a->len > b->len ? a->len : b->len;
  uint64_t carry = 0;
  for (int i = 0; i < n; i++) {
    uint64_t s = carry;
    if (i < a->len) s += a->w[i];
    if (i < b->len) s += b->w[i];
    r->w[i] = (uint32_t)s;
    carry = s >> 32;
  }
  r->w[n] = (uint32_t)carry;
  r->len = n + 1;
  bn_trim(r);
}

void bn_sub(bn* r, const bn* a, const bn* b) {
  uint32_t borrow = 0;
  for (int i = 0; i < a->len; i++) {
    uint64_t bi = (i < b->len ? (uint64_t)b->w[i] : 0u) + borrow;
    uint64_t ai = a->w[i];
    r->w[i] = (uint32_t)(ai - bi);
    borrow = ai < bi ? 1u : 0u;
  }
  r->len = a->len;
  bn_trim(r);
}

void bn_add_u32(bn* r, const bn* a, uint32_t v) {
  bn t;
  bn_set_u64(&t, v);
  bn_add(r, a, &t);
}

void bn_sub_u32(bn* r, const bn* a, uint32_t v) {
  bn t;
  bn_set_u64(&t, v);
  bn_sub(r, a, &t);
}

void bn_mul(bn* r, const bn* a, const bn* b) {
  static __thread bn t; /* r may alias a or b */
  int n = a->len + b->len;
  for (int i = 0; i < n; i++) t.w[i] = 0;
  for (int i = 0; i < a->len; i++) {
    uint64_t carry = 0;
    for (int j = 0; j < b->len; j++) {
      uint64_t p = (uint64_t)a->w[i] * b->w[j] + t.w[i + j] + carry;
      t.w[i + j] = (uint32_t)p;
      carry = p >> 32;
    }
    t.w[i + b->len] = (uint32_t)carry;
  }
  t.len = n;
  bn_trim(&t);
  bn_copy(r, &t);
}

/* Division by one word. */
static void bn_divmod_small(const bn* u, uint32_t v, bn* q, bn* r) {
  bn qq;
  uint64_t rem = 0;
  for (int i = u->len - 1; i >= 0; i--) {
    uint64_t cur = (rem << 32) | u->w[i];
    qq.w[i] = (uint32_t)(cur / v);
    rem = cur % v;
  }
  qq.len = u->len;
  bn_trim(&qq);
  if (q) bn_copy(q, &qq);
  if (r) bn_set_u64(r, rem);
}

/*
 * Knuth, TAOCP vol. 2, 4.3.1, Algorithm D: long division of an (m+n)-word
 * dividend by an n-word divisor (n >= 2), one quotient word per step, with
 * the divisor normalised so that its top bit is set.
 */
void bn_divmod(const bn* u, const bn* v, bn* q, bn* r) {
  if (v->len == 0) return; /* division by zero: caller's error */
  if (bn_cmp(u, v) < 0) {
    bn tmp;
    bn_copy(&tmp, u);
    if (q) bn_zero(q);
    if (r) bn_copy(r, &tmp);
    return;
  }
  if (v->len == 1) {
    bn_divmod_small(u, v->w[0], q, r);
    return;
  }
  int n = v->len, m = u->len - v->len;
  /* D1: normalise so that the divisor's leading word has its top bit set */
  int s = 0;
  uint32_t top = v->w[n - 1];
  while (!(top & 0x80000000u)) { top <<= 1; s++; }
  static __thread uint32_t vn[BN_MAX], un[BN_MAX + 1];
  for (int i = n - 1; i > 0; i--)
    vn[i] = s ? (v->w[i] << s) | (v->w[i - 1] >> (32 - s)) : v->w[i];
  vn[0] = v->w[0] << s;
  un[m + n] = s ? u->w[m + n - 1] >> (32 - s) : 0u;
  for (int i = m + n - 1; i > 0; i--)
    un[i] = s ? (u->w[i] << s) | (u->w[i - 1] >> (32 - s)) : u->w[i];
  un[0] = u->w[0] << s;
  bn qq;
  /* D2..D7: one quotient word per position, most significant first */
  for (int j = m; j >= 0; j--) {
    /* D3: estimate the quotient word from the top two dividend words */
    uint64_t num = ((uint64_t)un[j + n] << 32) | un[j + n - 1];
    uint64_t qhat = num / vn[n - 1];
    uint64_t rhat = num % vn[n - 1];
    while (qhat > 0xffffffffull || qhat * vn[n - 2] > ((rhat << 32) | un[j + n - 2])) {
      qhat--;
      rhat += vn[n - 1];
      if (rhat > 0xffffffffull) break;
    }
    /* D4: subtract qhat * divisor from the current dividend window */
    uint64_t carry = 0;
    uint32_t borrow = 0;
    for (int i = 0; i < n; i++) {
      uint64_t p = qhat * vn[i] + carry;
      carry = p >> 32;
      uint64_t sub = (uint64_t)(uint32_t)p + borrow;
      uint64_t cur = un[i + j];
      un[i + j] = (uint32_t)(cur - sub);
      borrow = cur < sub ? 1u : 0u;
    }
    uint64_t sub = carry + borrow;
    uint64_t cur = un[j + n];
    un[j + n] = (uint32_t)(cur - sub);
    int negative = cur < sub;
    /* D5/D6: the estimate was one too large: add the divisor back */
    if (negative) {
      qhat--;
      uint64_t c = 0;
      for (int i = 0; i < n; i++) {
        uint64_t t = (uint64_t)un[i + j] + vn[i] + c;
        un[i + j] = (uint32_t)t;
        c = t >> 32;
      }
      un[j + n] = (uint32_t)(un[j + n] + c);
    }
    qq.w[j] = (uint32_t)qhat;
  }
  qq.len = m + 1;
  bn_trim(&qq);
  if (r) {
    /* D8: the remainder is the low n words, shifted back */
    for (int i = 0; i < n; i++)
      r->w[i] = s ? (un[i] >> s) | (un[i + 1] << (32 - s)) : un[i];
    r->len = n;
    bn_trim(r);
  }
  if (q) bn_copy(q, &qq);
}

void bn_mod(bn* r, const bn* a, const bn* m) { bn_divmod(a, m, 0, r); }

void bn_mulmod(bn* r, const bn* a, const bn* b, const bn* m) {
  bn t;
  bn_mul(&t, a, b);
  bn_mod(r, &t, m);
}

/* Left-to-right binary exponentiation: square, then multiply when the bit is 1. */
void bn_powmod(bn* r, const bn* b, const bn* e, const bn* m) {
  bn base, acc;
  bn_mod(&base, b, m);
  bn_set_u64(&acc, 1);
  bn_mod(&acc, &acc, m); /* m == 1 gives 0 */
  for (int i = bn_bitlen(e) - 1; i >= 0; i--) {
    bn_mulmod(&acc, &acc, &acc, m);
    if (bn_bit(e, i)) bn_mulmod(&acc, &acc, &base, m);
  }
  bn_copy(r, &acc);
}

void bn_gcd(bn* r, const bn* a, const bn* b) {
  bn x, y, t;
  bn_copy(&x, a);
  bn_copy(&y, b);
  while (!bn_is_zero(&y)) {
    bn_mod(&t, &x, &y);
    bn_copy(&x, &y);
    bn_copy(&y, &t);
  }
  bn_copy(r, &x);
}

/* Extended Euclid with the Bezout coefficient of a kept reduced mod m. */
int bn_modinv(bn* r, const bn* a, const bn* m) {
  bn r0, r1, t0, t1, q, tmp, prod;
  bn_copy(&r0, m);
  bn_mod(&r1, a, m);
  bn_zero(&t0);
  bn_set_u64(&t1, 1);
  while (!bn_is_zero(&r1)) {
    bn_divmod(&r0, &r1, &q, &tmp);
    bn_copy(&r0, &r1);
    bn_copy(&r1, &tmp);
    /* (t0, t1) <- (t1, t0 - q*t1 mod m) */
    bn_mulmod(&prod, &q, &t1, m);
    if (bn_cmp(&t0, &prod) >= 0) {
      bn_sub(&tmp, &t0, &prod);
    } else {
      bn_sub(&tmp, m, &prod);
      bn_add(&tmp, &tmp, &t0);
    }
    bn_copy(&t0, &t1);
    bn_copy(&t1, &tmp);
  }
  bn one;
  bn_set_u64(&one, 1);
  if (bn_cmp(&r0, &one) != 0) return 0;
  bn_copy(r, &t0);
  return 1;
}

void bn_lcm(bn* r, const bn* a, const bn* b) {
  bn g, q;
  bn_gcd(&g, a, b);
  bn_divmod(a, &g, &q, 0);
  bn_mul(r, &q, b);
}
