// pc2_batch.h -- internal structures of the batched private ADMM round
// (many edge nodes, mixed key sizes, one persistent launch per round).
//
// Every node's design block is orthonormal, so Bbar_k = rho/(1+rho) I is
// diagonal and Eq. (itq2) splits into 1 x 1 blocks: element i of node k needs
// only its own z_i, v_i, alpha-hat_i and b_i = Gamma2(Bbar_ii).  One element's
// whole round -- Gamma2 of z and -v (Eq. (et21)), two encryptions
// (Eq. (itq1), CRT form of Sec. IV-A), the aggregation z-hat (+) (-v)-hat
// (Definition 1), b_i (x) s-hat (+) alpha-hat (Definition 2, Eq. (itq2)), CRT
// decryption, the exact decode of Theorem 1 with N_k = 1, and Eqs. (ty32),
// (u78) -- then runs inside one group of lanes with no exchange between
// elements.
#pragma once
#include <cstddef>
#include <cstdint>

#include "pc2_params.h"

namespace pc2 {

constexpr int kBatchClasses = 5;  // key sizes 256, 512, 1024, 2048, 3072 bits (Lh = 8, 16, 32, 64, 96)
constexpr int kBatchLh[kBatchClasses] = {8, 16, 32, 64, 96};
// Lanes per element in the batched kernel: one lane up to 2048-bit keys (the
// CRT moduli are read from constant memory with compile-time offsets), four
// at 3072 bits (24 limbs per lane with the modulus segment in registers), so
// that every class fits the kernel's register budget of three CTAs per SM.
constexpr int batch_lanes(int Lh) { return Lh == 96 ? 4 : 1; }
constexpr int batch_class(int Lh) {
  return Lh == 8 ? 0 : Lh == 16 ? 1 : Lh == 32 ? 2 : Lh == 64 ? 3 : Lh == 96 ? 4 : -1;
}

// Everything the kernel needs about one key, in device memory.
template <int Lh>
struct BatchKey {
  EncCrtParams<Lh> enc;    // p^2, q^2 constants, exponents n mod p(p-1), n mod q(q-1), n, p^2, (p^2)^-1 R mod q^2
  DecParams<Lh> dec;       // exponents p-1, q-1, p, q, L_p / L_q constants, Garner constant
  ModConst<2 * Lh> n2;     // n^2 (aggregation and scaling)
};

struct BatchNode {
  uint64_t elem0;   // global index of the node's first element
  uint64_t ct_off;  // word offset of the node's tiled ciphertexts in each ciphertext pool
  uint32_t count;   // N_k
  uint32_t cls;     // key class (index into kBatchLh)
};

// One work item: up to (128 / lanes) consecutive elements of one node.
struct BatchItem {
  uint32_t node;
  uint32_t first;   // index of the first element inside the node
  uint32_t count;
  uint32_t cls;
};

// Device-side control words of the persistent launch.
struct BatchCtl {
  uint32_t next;    // next unclaimed work item
  uint32_t done;    // CTAs finished in this launch
  uint32_t round;   // ADMM round t of the next launch (r-stream ids (t << 8) | kind)
  uint32_t pad_;
};

struct BatchParams {
  const void* key[kBatchClasses];  // BatchKey<Lh>* per class (null when absent)
  int tabw[kBatchClasses];         // words per group of the window-table region, per class
  const BatchNode* nodes;
  const BatchItem* items;
  uint32_t nitems;
  int dry;                         // 1: compute but write no state (timing by the autotuner)
  BatchCtl* ctl;
  const uint64_t* b;               // Gamma2(Bbar_ii), per element
  const uint32_t* alpha_hat;       // ciphertext pools (tiled per node, n^2 words per element)
  uint32_t* zhat;
  uint32_t* vhat;
  uint32_t* xhat;
  double* x;
  double* z;
  double* v;
  uint32_t* scratch;
  size_t cta_words;                // scratch words owned by one CTA
  int* status;
  uint64_t seed;
  double zmin, scale, qmax, kappa, inv_s2;
  long long mS, S;
};

// Moduli (p^2, q^2) and primes (p, q) of the classes run with one lane per
// element, copied to constant memory before each launch.
struct BatchConstMods {
  uint32_t m8[2][8];
  uint32_t m16[2][16];
  uint32_t m32[2][32];
  uint32_t m64[2][64];
  uint32_t h8[2][4];
  uint32_t h16[2][8];
  uint32_t h32[2][16];
  uint32_t h64[2][32];
};

int launch_batch_round(const BatchParams& P, const BatchConstMods* d_mods, size_t smem, int grid, cudaStream_t st);
// Resident CTAs per SM of the batched kernel with `smem` bytes of dynamic shared memory.
int batch_blocks_per_sm(size_t smem);
// Per-element decode and z/v update of the plain per-node path (N_k = 1 blocks).
int launch_batch_update(const uint32_t* D, int Lh, size_t n, const uint64_t* zq, const uint64_t* vq,
                        const uint64_t* b, long long mS, long long S, double inv_s2, double kappa, double* x,
                        double* z, double* v, int* status, uint32_t* round_ctr, int sms, cudaStream_t st);

}  // namespace pc2
