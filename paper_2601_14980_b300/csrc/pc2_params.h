// pc2_params.h -- kernel-parameter blocks and limits shared by the host
// launchers and the CUDA kernels of libpc2.
//
// Everything a kernel needs about a key travels BY VALUE in its parameter
// block (constant bank 0), so the modulus words become immediate operands of
// the multiply-add instructions and concurrent launches with different keys
// never share mutable state.
#pragma once
#include <cstdint>

namespace pc2 {

constexpr int kTile = 32;          // elements per tile of the interleaved layout
constexpr int kMaxSched = 1024;    // sliding-window steps for one exponent
constexpr int kMaxSchedHalf = 512; // per-prime decryption exponents (p-1, q-1)
constexpr int kMaxWin = 6;         // largest window width
constexpr int kMaxGroups = 32;     // operands of one hom_sum launch

// One Montgomery modulus N of L 32-bit limbs, R = 2^(32L).
template <int L>
struct ModConst {
  uint32_t n[L];   // N, little-endian words
  uint32_t r1[L];  // R mod N (Montgomery form of 1)
  uint32_t r2[L];  // R^2 mod N
  uint32_t r3[L];  // R^3 mod N
  uint32_t np;     // -N^{-1} mod 2^32
  uint32_t pad_[3];
};

// A fixed exponent as a left-to-right sliding-window schedule.  Step 0 loads
// table entry idx0; every later step squares `nsq` times and, when idx >= 0,
// multiplies by table entry idx (odd powers base^(2*idx+1)).
// Encoding: step = (nsq << 8) | (idx + 1).
template <int MAXS>
struct Sched {
  uint16_t step[MAXS];
  int32_t nsteps;
  int32_t w;          // window width (table of 2^(w-1) odd powers)
  int32_t montmuls;   // Montgomery products the schedule costs (table included)
  int32_t pad_;
};

// Public-key encryption mod n^2 (L2 = limbs of n^2).
template <int L2>
struct EncPubParams {
  ModConst<L2> m;          // modulus n^2
  Sched<kMaxSched> e;      // exponent n
  uint32_t nwords[L2 / 2]; // n (for 1 + m*n)
  uint64_t seed;
  uint64_t e0;             // global index of element 0 (counter of the r draw)
  uint32_t stream;
  int32_t mwords;          // words per plaintext: 2 (uint64 input) or L2/2 (wide, tiled input)
};

// r^n mod h^2 for one prime h of the key (h = p or q, h' the other one)
// without the full power by n mod h(h-1).  Since h | n, r^n mod h^2 depends
// on r mod h only, and r^h mod h^2 is the Teichmuller representative of
// r mod h (the unique (h-1)-th root of unity mod h^2 congruent to it); so
// r^n = (r^h)^(h') is the representative of s = r^(h' mod (h-1)) mod h, which
// is s^h mod h^2.  One power mod h (half width) by an exponent below h and
// one power mod h^2 by h replace one power mod h^2 by a full-width exponent.
template <int Lh>
struct LiftConst {
  ModConst<Lh / 2> h;          // the prime h, R_h = 2^(16 Lh)
  Sched<kMaxSchedHalf> e1;     // h' mod (h - 1)
  Sched<kMaxSchedHalf> e2;     // h
  uint32_t lift[Lh];           // R_h^3 mod h^2: Montgomery product with s R_h gives s R mod h^2
};

// The lifted route needs at least two limbs per lane at half width.
template <int Lh, int T>
constexpr bool lift_route() { return (Lh / 2) / T >= 2; }

// Key-owner encryption through CRT mod p^2 and q^2 (Lh = limbs of n = limbs of p^2).
// When round_ptr is set the r-stream id is (*round_ptr << 8) | kind, read on
// the device (so a captured ADMM round can be replayed round after round).
template <int Lh>
struct EncCrtParams {
  ModConst<Lh> mp, mq;       // p^2, q^2
  Sched<kMaxSched> ep, eq;   // n mod p(p-1), n mod q(q-1) (direct route)
  LiftConst<Lh> lp, lq;      // lifted route mod p^2, q^2 (window widths <= max(ep.w, eq.w))
  uint32_t nwords[Lh];       // n
  uint32_t p2[Lh];           // p^2 (for the recombination product)
  uint32_t pinv2R[Lh];       // (p^-2 mod q^2) * R mod q^2
  uint64_t seed;
  uint64_t e0;
  uint32_t stream;
  int32_t mwords;
  const uint32_t* round_ptr;
  uint32_t kind;
  uint32_t kind2;  // elements e >= split form a second vector (split-halves kernel only):
  uint64_t split;  // r-stream kind2, counter e0 + (e - split), tiled output position base2 + (e - split)
  uint64_t base2;
};

// CRT decryption (Lh = limbs of n; p, q have Lh/2 limbs).
template <int Lh>
struct DecParams {
  ModConst<Lh> mp, mq;            // p^2, q^2
  Sched<kMaxSchedHalf> ep, eq;    // p-1, q-1
  uint32_t p[Lh / 2], q[Lh / 2];  // the primes
  uint32_t pnp, qnp;              // -p^-1, -q^-1 mod 2^32
  uint32_t hpR[Lh / 2];           // h_p * R_h mod p, h_p = (-q)^-1 mod p  (R_h = 2^(32 Lh/2))
  uint32_t hqR[Lh / 2];           // h_q * R_h mod q, h_q = (-p)^-1 mod q
  uint32_t pinvqR[Lh / 2];        // p^-1 * R_h mod q
  uint32_t pinvlo[Lh / 2];        // p^-1 mod 2^(32 Lh/2)
  uint32_t qinvlo[Lh / 2];        // q^-1 mod 2^(32 Lh/2)
};

// Ciphertext products and powers mod n^2.
template <int L2>
struct HomParams {
  ModConst<L2> m;
  uint32_t rk[L2];                     // R^k mod n^2 (fix-up after k-1 products)
  const uint32_t* src[kMaxGroups];     // hom_sum operands (tiled arrays)
  int32_t ngroups;
  int32_t w;                           // window width for hom_scal
};

// Encrypted matrix-vector product of Eq. (itq2):
// out_i = alpha_i * prod_j s_j^{b_ij} mod n^2, rows grouped by edge node.
template <int L2>
struct MatvecParams {
  ModConst<L2> m;
  int32_t c;       // bucket window (bits); 2^c buckets per row
  int32_t nwin;    // windows covering the widest b_ij
  int32_t ntiles;  // row tiles (a tile = one CTA's rows, all of one node)
  int32_t pad_;
};

// Kernel parameter blocks travel by value: at most 32764 bytes per launch.
static_assert(sizeof(EncCrtParams<128>) + 256 <= 32764, "encryption parameter block too large");
static_assert(sizeof(DecParams<128>) + 256 <= 32764, "decryption parameter block too large");
static_assert(sizeof(EncPubParams<256>) + 256 <= 32764, "encryption parameter block too large");
static_assert(sizeof(HomParams<256>) + 256 <= 32764, "homomorphic parameter block too large");

}  // namespace pc2
