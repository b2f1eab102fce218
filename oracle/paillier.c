/*
 * paillier.c -- CPU oracle for the Paillier layer of 3P-ADMM-PC2.
 *
 * TEST INFRASTRUCTURE ONLY (see bn.h).  Every function computes the plain
 * definition the paper states, with the schoolbook arithmetic of bn.c:
 *
 *   key derivation   Sec. III-B (key generation list): n = pq,
 *                    lambda = lcm(p-1, q-1), g in Z*_{n^2},
 *                    mu = L(g^lambda mod n^2)^{-1} mod n, L(x) = (x-1)/n
 *   encryption       Eq. (itq1): c = g^m * r^n mod n^2
 *   decryption       Sec. III-C: m = L(c^lambda mod n^2) * mu mod n
 *   addition (+)     Definition 1, Eq. (headd): c1 * c2 mod n^2
 *   scaling (x)      Definition 2, Eq. (hemul): c^k mod n^2
 *   matrix (x)       Eq. (ldofi2)/(itq2) with Definition 2 applied row by
 *                    row: out_i = alpha_i * prod_j s_j^{K_ij} mod n^2
 *
 * The random r of Eq. (itq1) is an input.  r_raw() below is the counter-based
 * draw both sides implement from the published Philox4x32-10 definition
 * (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11): a (words)-word integer whose word 4j+i is output i of the block
 * cipher applied to counter (j, e_lo, e_hi, stream) under key (seed_lo,
 * seed_hi).  r = r_raw mod n.
 *
 * Numbers cross this interface as little-endian 32-bit word arrays of a
 * stated length.
 */
#include "bn.h"
#include <stddef.h>
#include <stdint.h>

/* ---- Philox4x32-10 (SC'11, Sec. 4.2 and its published constants) ---- */

static uint32_t mulhi32(uint32_t a, uint32_t b) { return (uint32_t)(((uint64_t)a * b) >> 32); }

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u; /* round multipliers */
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u; /* Weyl key increments */
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; round++) {
    if (round > 0) { k0 += W0; k1 += W1; }
    uint32_t hi0 = mulhi32(M0, c0), lo0 = M0 * c0;
    uint32_t hi1 = mulhi32(M1, c2), lo1 = M1 * c2;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void orc_r_raw(uint64_t seed, uint32_t stream, uint64_t e, int words, uint32_t* out) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int j = 0; 4 * j < words; j++) {
    uint32_t ctr[4] = {(uint32_t)j, (uint32_t)e, (uint32_t)(e >> 32), stream};
    uint32_t blk[4];
    orc_philox4x32_10(ctr, key, blk);
    for (int i = 0; i < 4 && 4 * j + i < words; i++) out[4 * j + i] = blk[i];
  }
}

/* ---- plain big-integer entry points used by the tests ---- */

int orc_powmod(const uint32_t* b, int bl, const uint32_t* e, int el, const uint32_t* m, int ml, uint32_t* out) {
  bn B, E, M, R;
  bn_from_words(&B, b, bl);
  bn_from_words(&E, e, el);
  bn_from_words(&M, m, ml);
  if (bn_is_zero(&M)) return -1;
  bn_powmod(&R, &B, &E, &M);
  bn_to_words(&R, out, ml);
  return 0;
}

int orc_mul(const uint32_t* a, int al, const uint32_t* b, int bl, uint32_t* out /* al+bl */) {
  bn A, B, R;
  bn_from_words(&A, a, al);
  bn_from_words(&B, b, bl);
  bn_mul(&R, &A, &B);
  bn_to_words(&R, out, al + bl);
  return 0;
}

int orc_divmod(const uint32_t* u, int ul, const uint32_t* v, int vl, uint32_t* q /* ul */, uint32_t* r /* vl */) {
  bn U, V, Q, R;
  bn_from_words(&U, u, ul);
  bn_from_words(&V, v, vl);
  if (bn_is_zero(&V)) return -1;
  bn_divmod(&U, &V, &Q, &R);
  bn_to_words(&Q, q, ul);
  bn_to_words(&R, r, vl);
  return 0;
}

int orc_modinv(const uint32_t* a, int al, const uint32_t* m, int ml, uint32_t* out) {
  bn A, M, R;
  bn_from_words(&A, a, al);
  bn_from_words(&M, m, ml);
  if (!bn_modinv(&R, &A, &M)) return -1;
  bn_to_words(&R, out, ml);
  return 0;
}

/* ---- Paillier (Sec. III-B/III-C of the paper) ---- */

/* L(x) = (x - 1) / n */
static void paillier_L(bn* out, const bn* x, const bn* n) {
  bn t;
  bn_sub_u32(&t, x, 1);
  bn_divmod(&t, n, out, 0);
}

/*
 * Key derivation from the primes.  Writes n (nw words), n^2 (2nw),
 * lambda (nw), mu (nw).  g is an input (the paper allows any g in Z*_{n^2}).
 * Returns 0, or -1 when mu does not exist (g not a valid base).
 */
int orc_paillier_derive(const uint32_t* p, const uint32_t* q, int pw, const uint32_t* g, int gw, int nw, uint32_t* n_out,
                        uint32_t* n2_out, uint32_t* lambda_out, uint32_t* mu_out) {
  bn P, Q, N, N2, G, P1, Q1, LAM, X, LX, MU;
  bn_from_words(&P, p, pw);
  bn_from_words(&Q, q, pw);
  bn_mul(&N, &P, &Q);
  bn_mul(&N2, &N, &N);
  bn_from_words(&G, g, gw);
  bn_sub_u32(&P1, &P, 1);
  bn_sub_u32(&Q1, &Q, 1);
  bn_lcm(&LAM, &P1, &Q1);
  bn_powmod(&X, &G, &LAM, &N2);
  paillier_L(&LX, &X, &N);
  if (!bn_modinv(&MU, &LX, &N)) return -1;
  bn_to_words(&N, n_out, nw);
  bn_to_words(&N2, n2_out, 2 * nw);
  bn_to_words(&LAM, lambda_out, nw);
  bn_to_words(&MU, mu_out, nw);
  return 0;
}

/* Eq. (itq1): c = g^m * r^n mod n^2, for count messages (each mw words), r (rw words each). */
int orc_paillier_encrypt(const uint32_t* n, int nw, const uint32_t* g, const uint32_t* m, int mw, const uint32_t* r, int rw,
                         int count, uint32_t* c /* count * 2nw */) {
  bn N, N2, G, M, R, GM, RN, C;
  bn_from_words(&N, n, nw);
  bn_mul(&N2, &N, &N);
  bn_from_words(&G, g, 2 * nw);
  for (int i = 0; i < count; i++) {
    bn_from_words(&M, m + (size_t)i * mw, mw);
    bn_from_words(&R, r + (size_t)i * rw, rw);
    bn_powmod(&GM, &G, &M, &N2);
    bn_powmod(&RN, &R, &N, &N2);
    bn_mulmod(&C, &GM, &RN, &N2);
    bn_to_words(&C, c + (size_t)i * 2 * nw, 2 * nw);
  }
  return 0;
}

/* Sec. III-C: m = L(c^lambda mod n^2) * mu mod n. */
int orc_paillier_decrypt(const uint32_t* n, int nw, const uint32_t* lambda, const uint32_t* mu, const uint32_t* c, int count,
                         uint32_t* m /* count * nw */) {
  bn N, N2, LAM, MU, C, X, LX, M;
  bn_from_words(&N, n, nw);
  bn_mul(&N2, &N, &N);
  bn_from_words(&LAM, lambda, nw);
  bn_from_words(&MU, mu, nw);
  for (int i = 0; i < count; i++) {
    bn_from_words(&C, c + (size_t)i * 2 * nw, 2 * nw);
    bn_powmod(&X, &C, &LAM, &N2);
    paillier_L(&LX, &X, &N);
    bn_mulmod(&M, &LX, &MU, &N);
    bn_to_words(&M, m + (size_t)i * nw, nw);
  }
  return 0;
}

/* Definition 1 applied over groups: out_i = prod_{g < groups} c[g*count + i] mod n^2. */
int orc_hom_sum(const uint32_t* n2, int cw, const uint32_t* c, int groups, int count, uint32_t* out) {
  bn N2, ACC, X;
  bn_from_words(&N2, n2, cw);
  for (int i = 0; i < count; i++) {
    bn_set_u64(&ACC, 1);
    for (int g = 0; g < groups; g++) {
      bn_from_words(&X, c + ((size_t)g * count + i) * cw, cw);
      bn_mulmod(&ACC, &ACC, &X, &N2);
    }
    bn_to_words(&ACC, out + (size_t)i * cw, cw);
  }
  return 0;
}

/* Definition 2: out_i = c_i^{k_i} mod n^2 with 64-bit scalars. */
int orc_hom_scal(const uint32_t* n2, int cw, const uint32_t* c, const uint64_t* k, int count, uint32_t* out) {
  bn N2, C, K, R;
  bn_from_words(&N2, n2, cw);
  for (int i = 0; i < count; i++) {
    bn_from_words(&C, c + (size_t)i * cw, cw);
    bn_set_u64(&K, k[i]);
    bn_powmod(&R, &C, &K, &N2);
    bn_to_words(&R, out + (size_t)i * cw, cw);
  }
  return 0;
}

/* Eq. (itq2): out_i = alpha_i * prod_j s_j^{K[i*cols+j]} mod n^2 (Definitions 1 and 2 row by row). */
int orc_hom_matvec(const uint32_t* n2, int cw, const uint32_t* alpha, const uint32_t* s, const uint64_t* K, int rows,
                   int cols, uint32_t* out) {
  bn N2, ACC, S, E, P;
  bn_from_words(&N2, n2, cw);
  for (int i = 0; i < rows; i++) {
    bn_from_words(&ACC, alpha + (size_t)i * cw, cw);
    for (int j = 0; j < cols; j++) {
      bn_from_words(&S, s + (size_t)j * cw, cw);
      bn_set_u64(&E, K[(size_t)i * cols + j]);
      bn_powmod(&P, &S, &E, &N2);
      bn_mulmod(&ACC, &ACC, &P, &N2);
    }
    bn_to_words(&ACC, out + (size_t)i * cw, cw);
  }
  return 0;
}
