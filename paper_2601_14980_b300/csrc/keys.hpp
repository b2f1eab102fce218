// keys.hpp -- host key object of libpc2 and the builders of the kernels'
// parameter blocks.
#pragma once
#include <cstdint>
#include <memory>
#include <vector>

#include "hostbn.hpp"
#include "pc2_params.h"

struct pc2_key {
  int nbits = 0;   // bits of n (multiple of 64)
  int Lh = 0;      // limbs of n (= limbs of p^2)
  bool priv = false;
  pc2::Big n, n2, lambda, mu;  // g = n + 1
  pc2::Big p, q;               // p < q (private keys)
};

namespace pc2 {

bool supported_nbits(int nbits);
bool probable_prime(const Big& x, int rounds, uint64_t seed);
int key_from_primes(const Big& p, const Big& q, pc2_key** out);

// Sliding-window schedule of exponent E with window width w (0: pick the
// width in 3..6 that needs the fewest products).  False if it does not fit.
template <int MAXS>
bool build_sched(const Big& E, int w, Sched<MAXS>& out);

template <int L>
void fill_mod(ModConst<L>& m, const Big& N);

// Parameter blocks (w = 0: automatic window).
template <int Lh> int make_enc_crt(const pc2_key& k, int w, EncCrtParams<Lh>& P);
template <int L2> int make_enc_pub(const pc2_key& k, int w, EncPubParams<L2>& P);
template <int Lh> int make_dec(const pc2_key& k, int w, DecParams<Lh>& P);
template <int L2> int make_hom(const pc2_key& k, int w, int ngroups, HomParams<L2>& P);

// The decryption parameter block of a key from the per-key host cache
// (built on first use; automatic window).
template <int Lh> std::shared_ptr<DecParams<Lh>> dec_params(const pc2_key* k, int* rc);
// The key-owner encryption block, likewise (automatic window).
template <int Lh> std::shared_ptr<EncCrtParams<Lh>> enc_params(const pc2_key* k, int* rc);

}  // namespace pc2
