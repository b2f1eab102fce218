/*
 * bn.h -- plain multi-precision unsigned integers for the CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This directory is the independent, slow,
 * obviously-correct reference that the CUDA library is checked against.
 * Only tests, the smoke check and the benchmark's CPU-baseline leg may use
 * it; the library never links, loads or imports anything from here.
 *
 * Numbers are little-endian arrays of 32-bit words with an explicit length.
 * Algorithms are the textbook ones: schoolbook multiplication, Knuth's
 * Algorithm D for division (TAOCP vol. 2, 4.3.1), left-to-right binary
 * exponentiation, Euclid's algorithm for gcd and inverses.  Nothing here
 * is shared with the CUDA path (which uses Montgomery arithmetic).
 */
#ifndef ORACLE_BN_H
#define ORACLE_BN_H
#include <stdint.h>

#define BN_MAX 640 /* words: room for products of two 8192-bit numbers */

typedef struct {
  int len;            /* significant words; w[len-1] != 0 unless len == 0 */
  uint32_t w[BN_MAX];
} bn;

void bn_zero(bn* a);
void bn_set_u64(bn* a, uint64_t v);
void bn_from_words(bn* a, const uint32_t* w, int n);
void bn_to_words(const bn* a, uint32_t* w, int n); /* zero-padded; n >= a->len */
void bn_copy(bn* dst, const bn* src);
int bn_is_zero(const bn* a);
int bn_cmp(const bn* a, const bn* b);
int bn_bitlen(const bn* a);
int bn_bit(const bn* a, int i);
void bn_add(bn* r, const bn* a, const bn* b);
void bn_sub(bn* r, const bn* a, const bn* b); /* requires a >= b */
void bn_add_u32(bn* r, const bn* a, uint32_t v);
void bn_sub_u32(bn* r, const bn* a, uint32_t v); /* requires a >= v */
void bn_mul(bn* r, const bn* a, const bn* b);
void bn_divmod(const bn* u, const bn* v, bn* q, bn* r); /* q or r may be NULL */
void bn_mod(bn* r, const bn* a, const bn* m);
void bn_mulmod(bn* r, const bn* a, const bn* b, const bn* m);
void bn_powmod(bn* r, const bn* b, const bn* e, const bn* m);
void bn_gcd(bn* r, const bn* a, const bn* b);
int bn_modinv(bn* r, const bn* a, const bn* m); /* returns 0 if no inverse */
void bn_lcm(bn* r, const bn* a, const bn* b);

#endif
