/*
 * pc2.h -- C ABI of libpc2: batched Paillier encryption, decryption and
 * homomorphic aggregation on one NVIDIA B300 (sm_103a), the data-parallel hot
 * path of 3P-ADMM-PC2 (arXiv 2601.14980).
 *
 * Conventions (every entry point):
 *  - Returns PC2_OK (0) or a negative PC2_E* code.  Argument errors are
 *    reported at the call; errors found on the device (a plaintext >= n, a
 *    quantizer input outside its range) set bits in the context's status
 *    word, read and cleared by pc2_ctx_status().
 *  - Pointers named d_* are DEVICE pointers owned by the caller (for example
 *    from torch tensors); h_* are host pointers.  Opaque objects (pc2_ctx,
 *    pc2_key) are owned by the library and freed by their *_destroy call.
 *  - Work is enqueued on the caller's stream and returns immediately.  Calls
 *    that share one pc2_ctx must be ordered on one stream (they share its
 *    scratch memory); use one context per concurrent stream.
 *  - Big integers are little-endian arrays of 32-bit words.  Device vectors
 *    of big integers use the TILED layout: 32-element tiles, each stored as
 *    (limbs/4) slabs of 32 x 16-byte vectors; word j of element e is at
 *        ((e/32) * (limbs/4) + j/4) * 128 + (e%32) * 4 + j%4.
 *    A tiled buffer of `count` elements holds pc2_tiled_words(count, limbs)
 *    words.  pc2_pack / pc2_unpack convert from / to the canonical layout
 *    (element e at words [e*limbs, (e+1)*limbs)).
 *  - Key sizes: n of 256, 512, 1024, 2048, 3072 or 4096 bits (the paper's
 *    evaluation uses 1024, 2048 and 4096).  Plaintexts have nbits/32 limbs,
 *    ciphertexts nbits/16 limbs.  The batched round (pc2_batch_*) takes the
 *    five sizes up to 3072 bits and the server 512- and 2048-bit keys (other
 *    sizes return PC2_EUNSUPPORTED); every other call takes all six.
 *  - Scratch: a context owns device scratch memory and grows it on the first
 *    call that needs more (cudaMalloc; synchronises the device).  Call
 *    pc2_ctx_reserve() first to avoid growth inside timed regions or stream
 *    capture.
 */
#ifndef PC2_H
#define PC2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* pc2_stream_t; /* a cudaStream_t; NULL = legacy default stream */

enum {
  PC2_OK = 0,
  PC2_EINVAL = -1,      /* bad argument (null pointer, unsupported size, ...) */
  PC2_ERANGE = -2,      /* a value outside the range the operation accepts */
  PC2_EKEY = -3,        /* private-key operation on a public key, or an invalid key */
  PC2_ENOMEM = -4,      /* device or host allocation failed */
  PC2_ECUDA = -5,       /* a CUDA call failed */
  PC2_ETIMEOUT = -6,    /* a bounded wait ran out */
  PC2_EMISSING = -7,    /* an expected input was not supplied */
  PC2_EUNSUPPORTED = -8 /* a configuration the library does not implement */
};

/* Status-word bits set by kernels (pc2_ctx_status). */
enum { PC2_ST_RANGE = 1, PC2_ST_QUANT = 2, PC2_ST_TIMEOUT = 4 };

typedef struct pc2_ctx pc2_ctx;
typedef struct pc2_key pc2_key;

const char* pc2_strerror(int code);

/* ---- context --------------------------------------------------------- */
/* Creates a context on CUDA device `device` (makes it current). */
int pc2_ctx_create(int device, pc2_ctx** out);
void pc2_ctx_destroy(pc2_ctx* ctx);
/* Grows the context's scratch to at least `bytes` now (synchronises). */
int pc2_ctx_reserve(pc2_ctx* ctx, size_t bytes);
/* Bytes of scratch currently held. */
size_t pc2_ctx_scratch_bytes(const pc2_ctx* ctx);
/* Synchronises `stream`, returns the PC2_ST_* bits raised since the last call in *bits, clears them. */
int pc2_ctx_status(pc2_ctx* ctx, pc2_stream_t stream, int* bits);
/* Forces the sliding-window width (3..6) of subsequent exponentiations; 0 = automatic. */
int pc2_ctx_set_window(pc2_ctx* ctx, int w);
/* Forces the lanes per element (1, 2, 4, 8) of the exponentiation kernels where
 * that count is built for the operand size; 0 = automatic: the autotuned
 * entry for the call's size class if any, else the lane count and split mode
 * with the lowest estimated time (the larger of a latency term -- waves of
 * resident element groups x halves run in sequence x (limbs per lane + 64)
 * per Montgomery row -- and an issue term the same for every lane count),
 * fitted to measured times: small batches get more lanes per element and
 * finish sooner, large ones run one lane per element. */
int pc2_ctx_set_lanes(pc2_ctx* ctx, int lanes);
/* Runs the two CRT halves of each element's exponentiations in parallel
 * (one half per two warps of a CTA, recombined after a block barrier):
 * mode 0 automatic (by the estimate of pc2_ctx_set_lanes), 1 never,
 * 2 always.  Results do not change. */
int pc2_ctx_set_split(pc2_ctx* ctx, int mode);
/* Engine of the full-width powers of key-owner encryption and CRT
 * decryption at 2048-bit n (Eq. (itq1), Sec. III-C): PC2_ENGINE_IMAD (the
 * one-kernel integer-pipe path), PC2_ENGINE_TC (the Montgomery products'
 * reductions on the tensor cores, see pc2_mont_sqr; three launches per call:
 * set-up, the powers, finish) or -1 automatic (the tensor cores from
 * PC2_TC_MIN_COUNT elements on).  Results do not change; other key sizes
 * always use the integer pipe.  PC2_EINVAL for another value. */
#define PC2_ENGINE_IMAD 0
#define PC2_ENGINE_TC 1
#define PC2_TC_MIN_COUNT 16384
int pc2_ctx_set_engine(pc2_ctx* ctx, int engine);
/* Stage timing of the tensor-core path (a measurement aid; the paper has no
 * counterpart).  With timing on, each tensor-core encryption or decryption
 * records CUDA events on its stream around its four launches, and
 * pc2_ctx_stage_ms writes the last such call's times in milliseconds to
 * h_ms[0..3]: set-up, power mod p^2, power mod q^2, finish (it waits for the
 * last event).  PC2_EINVAL unless the context's last encryption or
 * decryption ran, timed, on the tensor-core engine. */
int pc2_ctx_set_timing(pc2_ctx* ctx, int on);
int pc2_ctx_stage_ms(pc2_ctx* ctx, double* h_ms);
/* Squarings and general products of the full-width powers of one key-owner
 * encryption (op 0: the lifted route's powers by p and q, or the reduced
 * exponents) or decryption (op 2: by p - 1 and q - 1), tables included, and
 * the limbs of their modulus.  Keys up to 2048 bits. */
int pc2_key_power_counts(const pc2_key* key, int op, long* squarings, long* multiplies, int* limbs);
/* Autotuner: times every built lane count x split (on, off) x window
 * width (4..6) of key-owner encryption (ops bit 0) and/or decryption (bit 1)
 * on `count` elements (at most two resident waves of them) and records the
 * fastest for calls of the same size class (ceil(log2 count)) on this key
 * size in this context.  h_result (optional) receives (lanes, window, split)
 * per tuned op, in that order.  Allocates and frees temporary device
 * buffers; synchronises `stream`. */
int pc2_autotune(pc2_ctx* ctx, const pc2_key* key, size_t count, int ops, pc2_stream_t stream, int* h_result);

/* ---- keys (host) ------------------------------------------------------ *
 * Sec. III-B: n = pq, lambda = lcm(p-1, q-1), g = n + 1 (so g^m = 1 + mn and
 * mu = lambda^-1 mod n).  Key generation is deterministic in `seed`: primes of
 * nbits/2 bits with the top two bits set, from a Philox4x32-10 stream, sieved
 * and checked by 32 Miller-Rabin rounds. */
int pc2_keygen(int nbits, uint64_t seed, pc2_key** out);
/* A private key from given primes (each `words` words, equal bit length
 * nbits/2); rejects composites (Miller-Rabin), p == q, or gcd(n, lambda) != 1. */
int pc2_key_from_primes(const uint32_t* h_p, const uint32_t* h_q, int words, pc2_key** out);
/* A public copy (n, g only) of a key. */
int pc2_key_public(const pc2_key* key, pc2_key** out);
void pc2_key_destroy(pc2_key* key);
/* nbits and whether the key holds the private part. */
int pc2_key_info(const pc2_key* key, int* nbits, int* has_private);
/* Exports n (nbits/32 words); for private keys also p, q (p < q; nbits/64
 * words each), lambda and mu (nbits/32 words each).  Any pointer may be NULL. */
int pc2_key_export(const pc2_key* key, uint32_t* h_n, uint32_t* h_p, uint32_t* h_q, uint32_t* h_lambda, uint32_t* h_mu);
/* Montgomery products one call costs per element (for throughput accounting):
 * op 0 = pc2_encrypt (key owner, CRT), 1 = public encryption, 2 = decryption.
 * *montmuls receives the products of *limbs words, *montmuls_half those of
 * *limbs / 2 words (the half-width powers mod p and q of the key-owner
 * encryption as the one-lane kernels run it; 0 for ops 1 and 2).  The few
 * conversion products per element outside the powers are not counted. */
int pc2_key_cost(const pc2_ctx* ctx, const pc2_key* key, int op, long* montmuls, long* montmuls_half, int* limbs);

/* ---- layout ----------------------------------------------------------- */
size_t pc2_tiled_words(size_t count, int limbs);
int pc2_pack(pc2_ctx* ctx, const uint32_t* d_canon, size_t count, int limbs, uint32_t* d_tiled, pc2_stream_t stream);
int pc2_unpack(pc2_ctx* ctx, const uint32_t* d_tiled, size_t count, int limbs, uint32_t* d_canon, pc2_stream_t stream);

/* ---- Paillier ---------------------------------------------------------- *
 * Encryption, Eq. (itq1): c = g^m r^n mod n^2 with g = n + 1.  The random r of
 * element e (0-based in this call) is r_raw mod n, where r_raw is the
 * (nbits/32 + 2)-word integer whose word 4j+i is output i of Philox4x32-10
 * for counter (j, E_lo, E_hi, stream) and key (seed_lo, seed_hi), E = e0 + e.
 * (Only r mod n matters: (r + tn)^n = r^n mod n^2.)
 * d_m: `count` uint64 plaintexts.  d_ct: tiled, nbits/16 limbs.
 * With a private key the work runs through the CRT split of Sec. IV-A
 * (Lemmas 1-2, Eq. (gA-C-B)); with a public key directly mod n^2.  Both
 * give the same ciphertext. */
int pc2_encrypt(pc2_ctx* ctx, const pc2_key* key, const uint64_t* d_m, size_t count, uint64_t seed, uint32_t stream,
                uint64_t e0, uint32_t* d_ct, pc2_stream_t cstream);
/* As pc2_encrypt, plaintexts of full width: d_m tiled, nbits/32 limbs, each m < n
 * (m >= n raises PC2_ST_RANGE). */
int pc2_encrypt_wide(pc2_ctx* ctx, const pc2_key* key, const uint32_t* d_m, size_t count, uint64_t seed,
                     uint32_t stream, uint64_t e0, uint32_t* d_ct, pc2_stream_t cstream);
/* Public-key encryption mod n^2 even when the key is private (same result as pc2_encrypt). */
int pc2_encrypt_public(pc2_ctx* ctx, const pc2_key* key, const uint64_t* d_m, size_t count, uint64_t seed,
                       uint32_t stream, uint64_t e0, uint32_t* d_ct, pc2_stream_t cstream);
/* Decryption, Sec. III-C: m = L(c^lambda mod n^2) mu mod n, computed through
 * the CRT (m_p = L_p(c^(p-1) mod p^2) h_p mod p, likewise for q, then Garner).
 * d_ct: tiled, nbits/16 limbs; d_m: tiled, nbits/32 limbs.  PC2_EKEY for a public key. */
int pc2_decrypt(pc2_ctx* ctx, const pc2_key* key, const uint32_t* d_ct, size_t count, uint32_t* d_m,
                pc2_stream_t cstream);
/* Definition 1 (Eq. (headd)): d_out = d_a * d_b mod n^2 (encrypts a + b mod n). */
int pc2_hom_add(pc2_ctx* ctx, const pc2_key* key, const uint32_t* d_a, const uint32_t* d_b, size_t count,
                uint32_t* d_out, pc2_stream_t cstream);
/* Definition 1 over `groups` operands: d_out[i] = prod_g d_ct[g][i] mod n^2.
 * d_ct holds the groups back to back, each a tiled array of `count` ciphertexts
 * (group g starts at word g * pc2_tiled_words(count, nbits/16)). */
int pc2_hom_sum(pc2_ctx* ctx, const pc2_key* key, const uint32_t* d_ct, size_t groups, size_t count, uint32_t* d_out,
                pc2_stream_t cstream);
/* Definition 2 (Eq. (hemul)): d_out[i] = d_ct[i]^k[i] mod n^2 (encrypts k m mod n). */
int pc2_hom_scal(pc2_ctx* ctx, const pc2_key* key, const uint32_t* d_ct, const uint64_t* d_k, size_t count,
                 uint32_t* d_out, pc2_stream_t cstream);
/* Definition 2 with a full-width scalar (k in Z_n, as Definition 2 states it):
 * d_out[i] = d_ct[i]^k[i] mod n^2, d_k a tiled array of `count` scalars of
 * nbits/32 limbs each (any k < 2^nbits).  Every element takes the same
 * number of window steps (fixed windows over all nbits bits; the context's
 * window width clamped to 4..6, else 5), so a short k costs as much as a long
 * one.  This is also the plain power mod n^2 by a full-width exponent. */
int pc2_hom_scal_wide(pc2_ctx* ctx, const pc2_key* key, const uint32_t* d_ct, const uint32_t* d_k, size_t count,
                      uint32_t* d_out, pc2_stream_t cstream);

/* ---- quantizer ------------------------------------------------------- *
 * Eq. (et21) with one public range [zmin, zmax] and scale S = 2^log2_scale
 * (Delta = S (zmax - zmin)): gamma 2 -> q = rint((u - zmin) S) in [0, Delta];
 * gamma 1 -> q = rint((u - zmin) S^2) in [0, Delta S]; negate = 1 quantizes -u.
 * IEEE double, round half to even, no contraction.  Out-of-range inputs are
 * clamped and raise PC2_ST_QUANT.  d_u: n doubles; d_q: n uint64. */
int pc2_quantize(pc2_ctx* ctx, const double* d_u, size_t n, double zmin, double zmax, int log2_scale, int gamma,
                 int negate, uint64_t* d_q, pc2_stream_t stream);

/* Inverse of pc2_quantize: u = q / S + zmin (gamma 2) or q / S^2 + zmin
 * (gamma 1), IEEE double (exact whenever u needs at most 53 significant bits,
 * as the quantizer's outputs do).  d_q: n uint64; d_u: n doubles. */
int pc2_dequantize(pc2_ctx* ctx, const uint64_t* d_q, size_t n, double zmin, int log2_scale, int gamma, double* d_u,
                   pc2_stream_t stream);
/* The exact decode of Theorem 1 for rows of an encrypted matvec (Eq. (itq2)
 * decrypted): with mS = zmin S (an integer),
 *   x_i = fl(D_i + mS S + 2 mS brow_i + mS asum_i + 2 mS^2 nk_i) / S^2,
 * D_i the decrypted integers (tiled, `limbs` words each, < 2^128), brow_i =
 * sum_j b_ij over the row, asum_i = sum_j a_j over its block (a_j = Gamma2(z_j)
 * + Gamma2(-v_j)), nk_i the block's column count.  PC2_ST_RANGE when a D_i is
 * 2^128 or more or the sum leaves 64 bits. */
int pc2_decode_matvec(pc2_ctx* ctx, const uint32_t* d_D, int limbs, size_t n, const long long* d_brow,
                      const unsigned long long* d_asum, const int* d_nk, double zmin, int log2_scale, double* d_x,
                      pc2_stream_t stream);
/* The master's update, Eqs. (ty32) and (u78), elementwise in IEEE double
 * without contraction: a = v_i + x_i, z_i = S_kappa(a) (a - kappa above kappa,
 * a + kappa below -kappa, else 0), v_i = a - z_i.  d_z and d_v are updated in
 * place; n < 2^31. */
int pc2_zv_update(pc2_ctx* ctx, const double* d_x, double* d_z, double* d_v, size_t n, double kappa,
                  pc2_stream_t stream);

/* ---- encrypted matrix-vector product ----------------------------------- *
 * Eq. (itq2) on one n x n block: out_i = alpha_i (+) sum_j K_ij (x) s_j =
 * alpha_i * prod_j s_j^{K_ij} mod n^2, by the bucket method of the ADMM
 * round (same kernels, same window choice).  d_alpha, d_s, d_out: n tiled
 * ciphertexts; d_K: n*n uint32, row-major, every K_ij < 2^kbits (kbits 1..32,
 * 0 = 32; higher bits are ignored).  Scratch from the context. */
int pc2_hom_matvec(pc2_ctx* ctx, const pc2_key* key, const uint32_t* d_alpha, const uint32_t* d_s, const uint32_t* d_K,
                   size_t n, int kbits, uint32_t* d_out, pc2_stream_t stream);

/* ---- 3P-ADMM-PC2 on one GPU (Algorithm 1) ------------------------------- *
 * The K edge nodes are segments of device vectors (node k owns elements
 * [N_0 + ... + N_{k-1}, ... + N_k)).  Inputs are the edge nodes' set-up
 * results of Sec. II: d_alpha = alpha_k = B_k A_k^T y (N doubles, node by node)
 * and d_Bbar = rho B_k, B_k = (A_k^T A_k + rho I)^-1 (sum N_k^2 doubles,
 * row-major per node, node by node).  pc2_admm_create quantizes them
 * (Gamma1(alpha), Gamma2(Bbar)), encrypts alpha (r-stream 0) and sets
 * x = z = v = 0, round 1.  One private round (pc2_admm_round):
 *   Gamma2(z), Gamma2(-v); z-hat, (-v)-hat = E(.) with r-streams
 *   (t << 8) | 1 and (t << 8) | 2 (t = round); s-hat = z-hat (+) (-v)-hat;
 *   x-hat_k = alpha-hat_k (+) Gamma2(Bbar_k) (x) s-hat_k (Eq. (itq2));
 *   D = decrypt(x-hat); x = exact decode of D; z = S_{lambda/rho}(v + x);
 *   v = v + x - z (Eqs. (ty32), (u78)).
 * The exact decode: with mS = zmin S (must be an integer),
 *   x_i = fl(D_i + mS S + 2 mS sum_j b_ij + mS sum_j a_j + 2 mS^2 N_k) / S^2,
 * a_j = Gamma2(z_j) + Gamma2(-v_j), b = Gamma2(Bbar_k): the float64 rounding
 * of alpha~ + Bbar~ w~ on the dequantized inputs (Theorem 1 written out).
 * The batched path (per_node = 0) runs all nodes in the same launches and
 * replays rounds 2.. as one CUDA graph; per_node = 1 launches each node's
 * encryption, aggregation, matvec and decryption separately. */
typedef struct {
  int nodes;             /* K */
  const int* node_sizes; /* host array of K sizes N_k */
  double lambda, rho;
  double zmin, zmax;     /* public quantization range */
  int log2_scale;        /* S = 2^log2_scale */
  uint64_t seed;         /* Philox key of the encryption randomness */
  int per_node;          /* 0: batched + CUDA graph; 1: one launch per node */
} pc2_admm_params;

typedef struct pc2_admm pc2_admm;
int pc2_admm_create(pc2_ctx* ctx, const pc2_key* key, const pc2_admm_params* params, const double* d_alpha,
                    const double* d_Bbar, pc2_admm** out, pc2_stream_t stream);
void pc2_admm_destroy(pc2_admm* admm);
/* x = z = v = 0, round counter 1 (synchronises `stream`). */
int pc2_admm_reset(pc2_admm* admm, pc2_stream_t stream);
/* `rounds` private rounds of Algorithm 1.  PC2_EMISSING, before any launch
 * and with x, z, v and the round counter unchanged, while an edge node is
 * marked absent (pc2_admm_set_node_present). */
int pc2_admm_round(pc2_admm* admm, int rounds, pc2_stream_t stream);
/* Failure detection on the host.  In every round of Algorithm 1 the master
 * needs each edge node's segment (its x-hat_k; Sec. V reports the waiting
 * between nodes).  The orchestrator that collects the segments marks node
 * `node` (0 <= node < K) absent (present = 0) when its segment has not
 * arrived, and present again when it has; pc2_admm_round refuses to run
 * while any node is absent.  All nodes start present.  PC2_EINVAL for a bad
 * node index. */
int pc2_admm_set_node_present(pc2_admm* admm, int node, int present);
/* `rounds` plaintext Dis-ADMM rounds (Eq. (sldo091), (ty32), (u78)) on the same state, FP64. */
int pc2_admm_round_plain(pc2_admm* admm, int rounds, pc2_stream_t stream);
/* Copies x, z, v (device, N doubles each; any may be NULL) and the next round number (host; synchronises). */
int pc2_admm_get(pc2_admm* admm, double* d_x, double* d_z, double* d_v, uint32_t* h_round, pc2_stream_t stream);
/* Restores a checkpoint: x, z, v and the next round number (>= 1). */
int pc2_admm_set(pc2_admm* admm, const double* d_x, const double* d_z, const double* d_v, uint32_t round,
                 pc2_stream_t stream);
/* Checkpoint to / from host memory: x, z, v (N doubles each) and the next
 * round number (synchronises the device). */
int pc2_admm_save(pc2_admm* admm, double* h_x, double* h_z, double* h_v, uint32_t* h_round);
int pc2_admm_load(pc2_admm* admm, const double* h_x, const double* h_z, const double* h_v, uint32_t round);
/* Device pointers of the last round's ciphertexts (tiled) and decrypted integers, and N. */
int pc2_admm_buffers(pc2_admm* admm, const uint32_t** zhat, const uint32_t** vhat, const uint32_t** xhat,
                     const uint32_t** alpha_hat, const uint32_t** D, int* N);
/* Form of the encrypted matvec: 0 automatic (windows spread over CTAs when
 * the row tiles alone would fill less than half of the GPU), 1 one CTA per
 * row tile, 2 every (row tile, bucket window) pair its own work item, then a
 * per-row combination.  Results do not change; the captured round graph is
 * rebuilt on the next round. */
int pc2_admm_set_matvec(pc2_admm* admm, int mode);
/* Bucket window c, windows per exponent, CTA row tiles of the matvec. */
int pc2_admm_info(const pc2_admm* admm, int* c, int* nwin, int* ntiles);

/* ---- batched rounds: many edge nodes, mixed key sizes ------------------ *
 * The batching form of Algorithm 1: K edge nodes of uneven sizes, each node
 * holding a key of one of up to five sizes (256 .. 3072-bit n; one key per
 * size), every node's design block orthonormal (A_k^T A_k = I), so that
 * B_k = I / (1 + rho), Bbar_k = rho / (1 + rho) I and Eq. (itq2) splits into
 * 1 x 1 blocks.  Inputs: d_alpha = alpha_k = A_k^T y / (1 + rho) and d_bdiag =
 * the diagonal of Bbar_k (N doubles each, node by node).  Element i of node k
 * then runs, per round t: Gamma2(z_i), Gamma2(-v_i); z-hat_i, (-v)-hat_i =
 * E_k(.) with r-streams (t << 8) | 1, (t << 8) | 2 and counter i (global
 * index); x-hat_i = alpha-hat_i (+) b_i (x) (z-hat_i (+) (-v)-hat_i) with
 * b_i = Gamma2(Bbar_ii); D_i = decrypt_k(x-hat_i); the exact decode with
 * N_k = 1: x_i = fl(D_i + mS S + 2 mS b_i + mS (a_z + a_v) + 2 mS^2) / S^2;
 * z_i = S_{lambda/rho}(v_i + x_i), v_i = v_i + x_i - z_i.  alpha-hat_i =
 * E_k(Gamma1(alpha_i)) with r-stream 0.
 * pc2_batch_round runs each round as ONE persistent launch over a work list
 * of element tiles ordered longest first, captured once as a CUDA graph and
 * replayed (a device round counter advances the r-streams); it uses constant
 * memory of the library, so one batched round at a time may run per device.
 * Nodes of a 2048-bit key that the tensor-core engine takes (PC2_TC_MIN_COUNT
 * elements or more with the engine automatic, any size with it forced to
 * PC2_ENGINE_TC; decided at pc2_batch_create) stay out of the work list: each
 * batched round runs them node by node, as below, before the launch.
 * pc2_batch_round_per_node runs the same round node by node through the
 * per-operation kernels (pc2_encrypt, pc2_hom_add, pc2_hom_scal,
 * pc2_decrypt) and gives bit-identical state.  Status bits: PC2_ST_QUANT
 * (a z or -v outside [zmin, zmax]), PC2_ST_RANGE (a decoded value outside
 * 64 bits). */
typedef struct {
  int nodes;                  /* K */
  const int* node_sizes;      /* host, K sizes N_k >= 1 */
  const int* node_key;        /* host, K indices into keys[] */
  int nkeys;
  const pc2_key* const* keys; /* private keys, pairwise different sizes */
  double lambda, rho;
  double zmin, zmax;          /* public quantization range */
  int log2_scale;             /* S = 2^log2_scale */
  uint64_t seed;              /* Philox key of the encryption randomness */
} pc2_batch_params;

typedef struct pc2_batch pc2_batch;
/* Quantizes and encrypts the inputs, builds the work list, x = z = v = 0,
 * round 1.  Device buffers are owned by the object. */
int pc2_batch_create(pc2_ctx* ctx, const pc2_batch_params* params, const double* d_alpha, const double* d_bdiag,
                     pc2_batch** out, pc2_stream_t stream);
void pc2_batch_destroy(pc2_batch* batch);
/* x = z = v = 0, round 1 (synchronises `stream`). */
int pc2_batch_reset(pc2_batch* batch, pc2_stream_t stream);
/* `rounds` rounds, one persistent launch each (CUDA graph). */
int pc2_batch_round(pc2_batch* batch, int rounds, pc2_stream_t stream);
/* `rounds` rounds of the plain per-node path on the same state. */
int pc2_batch_round_per_node(pc2_batch* batch, int rounds, pc2_stream_t stream);
/* Copies x, z, v (device, N doubles each; any may be NULL) and the next round (host; synchronises). */
int pc2_batch_get(pc2_batch* batch, double* d_x, double* d_z, double* d_v, uint32_t* h_round, pc2_stream_t stream);
/* Device pointer of node `node`'s tiled ciphertexts of the last round
 * (which: 0 alpha-hat, 1 z-hat, 2 (-v)-hat, 3 x-hat) and their limbs (2 L(n)). */
int pc2_batch_ciphertexts(pc2_batch* batch, int which, int node, const uint32_t** d_tiled, int* limbs);
/* Elements, work items, persistent grid and scratch bytes of the batched
 * launch (the work items leave out the tensor-core nodes). */
int pc2_batch_info(const pc2_batch* batch, size_t* elements, int* items, int* grid, size_t* scratch_bytes);
/* Autotuner: times the window width (4..6) of each key's exponent schedules
 * and the CTAs per SM (1..3) of the persistent launch on a sample of the work
 * list (sample_items; 0 = one wave) without changing the state, and keeps the
 * fastest.  h_result (optional, 6 ints): the window per key size (256, 512,
 * 1024, 2048, 3072 bits; 0 = absent) and the CTAs per SM.  Synchronises. */
int pc2_batch_tune(pc2_batch* batch, int sample_items, pc2_stream_t stream, int* h_result);

/* ---- serving: a request loop with continuous batching ------------------ *
 * A server owns one private key (512 or 2048-bit n) and a device arena for
 * the requests' buffers.  Callers (any thread) submit encrypt, decrypt and
 * aggregate requests with HOST buffers, which must stay valid (and, for
 * asynchronous copies, should be page-locked) until pc2_server_wait returns.
 *   PC2_OP_ENCRYPT   in: count uint64 plaintexts; out: tiled ciphertexts
 *                    (2 L(n) limbs); the result equals pc2_encrypt(.., seed,
 *                    stream, e0, ..) (key-owner CRT path).
 *   PC2_OP_DECRYPT   in: tiled ciphertexts; out: tiled plaintexts (L(n) limbs),
 *                    equal to pc2_decrypt.
 *   PC2_OP_AGGREGATE in: `groups` (2..32) tiled ciphertext arrays of `count`
 *                    elements, h_stride words apart (0: back to back,
 *                    pc2_tiled_words(count, 2 L(n)) words; a larger stride
 *                    takes the first `count` elements of longer arrays);
 *                    out: their product mod n^2, equal to pc2_hom_sum.
 * Mode 0 (continuous batching): a worker thread admits requests in arrival
 * order as arena space frees up (first fit; at most max_active at once),
 * copies their inputs in, and runs steps, each ONE persistent launch over
 * work items of every admitted request.  Lanes per element are chosen per
 * request and step: every encrypt/decrypt request starts at 8 lanes per CRT
 * half with the two halves in parallel, and while the step's threads exceed
 * one resident wave the request with the largest demand steps down to 2 and
 * 1 lanes per half, then one lane per element; requests of at most
 * small_request elements keep the 8-lane form.  A
 * step holds about step_budget one-lane encryption items per CTA; two steps
 * are in flight, so requests that arrive while others run join the next step
 * and their work
 * overlaps on the device.  Mode 1 (the plain per-request path): requests run
 * one at a time, in arrival order, through pc2_encrypt / pc2_decrypt /
 * pc2_hom_sum on the context (do not use that context from other threads
 * meanwhile).  Results are identical in both modes and do not depend on what
 * else runs.  Servers of the same key size share a constant-memory block: at
 * most one of them may have requests in flight at a time. */
enum { PC2_OP_ENCRYPT = 1, PC2_OP_DECRYPT = 2, PC2_OP_AGGREGATE = 3 };
typedef struct {
  size_t arena_bytes;    /* device bytes for the requests' buffers (admission limit) */
  int mode;              /* 0: continuous batching; 1: plain per-request path */
  int max_active;        /* requests admitted at once (0: 256) */
  size_t small_request;  /* requests of at most this many elements always get 8 lanes per CRT half (0: 4096) */
  double step_budget;    /* work per CTA and step, in one-lane encryption items (0: 1.0) */
} pc2_server_params;

typedef struct pc2_server pc2_server;
int pc2_server_create(pc2_ctx* ctx, const pc2_key* key, const pc2_server_params* params, pc2_server** out);
/* Finishes the requests already submitted, then frees everything. */
void pc2_server_destroy(pc2_server* server);
/* Queues a request; *ticket identifies it.  PC2_ENOMEM when its buffers can
 * never fit the arena. */
int pc2_server_submit(pc2_server* server, int op, const void* h_in, size_t count, int groups, size_t h_stride,
                      uint64_t seed, uint32_t stream, uint64_t e0, void* h_out, uint64_t* ticket);
/* Blocks until the request is done (its output is in h_out) or timeout_s
 * passes (PC2_ETIMEOUT; the ticket stays valid).  latency_s: submit to done.
 * Returns the request's status and forgets the ticket. */
int pc2_server_wait(pc2_server* server, uint64_t ticket, double timeout_s, double* latency_s);
/* Requests completed, steps launched, work items run, peak arena bytes in use. */
int pc2_server_stats(pc2_server* server, uint64_t* completed, uint64_t* steps, uint64_t* items, size_t* arena_peak);

/* ---- collaborative CRT split between the master and an edge node ---- *
 * Sec. IV-C, Algorithm 3: edge node k holds p^2 and phi(p^2) (sent once by
 * the master) and computes the p^2 half of the master's encryptions and the
 * residues mod p^2 of its own ciphertexts; the master computes the q^2
 * halves and recombines (Lemmas 1-2, Eq. (gA-C-B)).  The obfuscation O(.),
 * which the paper leaves undefined, is an additive mask: O(w) = w + kappa.
 * Exchange 1: the master sends O(w) (pc2_collab_mask) and the edge
 * returns c'_masked = g^(O(w) mod phi(p^2)) r^n mod p^2
 * (pc2_collab_edge_encrypt); the master removes the mask with
 * g^(phi(p^2) - kappa mod phi(p^2)) and forms E(w; r) (pc2_collab_master_
 * encrypt): the same ciphertext as pc2_encrypt with the same seed, stream
 * and counters.  For decryption the edge sends x-hat mod p^2
 * (pc2_collab_edge_reduce) and the master decrypts from it and its own
 * residue mod q^2 (pc2_collab_master_decrypt), as pc2_decrypt.
 *  - Keys of 256 to 2048 bits (PC2_EUNSUPPORTED otherwise); `key` must be
 *    private (PC2_EKEY).  The edge calls read only p^2, phi(p^2), n and the
 *    schedule of the power r^n mod p^2 from it.
 *  - Device vectors in the tiled layout: w uint64 plaintexts (quantized
 *    values, below 2^64); kappa, O(w) and the p^2 halves/residues L words
 *    (L = words of n); ciphertexts 2L words; plaintexts L words.
 *  - kappa must be below 2^(32 L) - 2^64 so that O(w) fits L words; a carry
 *    out raises PC2_ST_RANGE in the status word.
 *  - Asynchronous on `stream`; scratch from the context. */
int pc2_collab_mask(pc2_ctx* ctx, const pc2_key* key, const uint64_t* d_w, const uint32_t* d_kappa, size_t count,
                    uint32_t* d_ow, pc2_stream_t stream);
int pc2_collab_edge_encrypt(pc2_ctx* ctx, const pc2_key* key, const uint32_t* d_ow, size_t count, uint64_t seed,
                            uint32_t stream, uint64_t e0, uint32_t* d_cp, pc2_stream_t cstream);
int pc2_collab_master_encrypt(pc2_ctx* ctx, const pc2_key* key, const uint64_t* d_w, const uint32_t* d_kappa,
                              const uint32_t* d_cp, size_t count, uint64_t seed, uint32_t stream, uint64_t e0,
                              uint32_t* d_ct, pc2_stream_t cstream);
int pc2_collab_edge_reduce(pc2_ctx* ctx, const pc2_key* key, const uint32_t* d_ct, size_t count, uint32_t* d_cp,
                           pc2_stream_t cstream);
int pc2_collab_master_decrypt(pc2_ctx* ctx, const pc2_key* key, const uint32_t* d_ct, const uint32_t* d_cp,
                              size_t count, uint32_t* d_m, pc2_stream_t cstream);

/* ---- Montgomery squarings on the tensor cores (an experiment) ------- *
 * nsq Montgomery squarings of each element: y = x^(2^nsq) R^-(2^nsq - 1)
 * mod N, R = 2^(32 limbs), the dominant operation of the fixed-exponent
 * powers of Eq. (itq1) and Sec. III-C.  engine PC2_ENGINE_IMAD runs the
 * library's CIOS product on the integer pipe; PC2_ENGINE_TC computes the
 * product a a on the integer pipe and the reduction's two contractions with
 * the fixed modulus, m = (T mod R) N' mod R and m N, as f16 tcgen05.mma
 * over 8-bit digits (the paper's recasting of big-integer products as
 * low-bitwidth matrix operations, Alg. 2, done on B300's tensor cores).  Both
 * give the same integers.
 *  - h_n: N, `limbs` little-endian words in host memory, odd; limbs = 64
 *    (2048-bit N) only (PC2_EUNSUPPORTED otherwise).
 *  - d_x, d_y: device, tiled layout of `limbs` words per element, x < N
 *    (not checked); d_y may equal d_x.
 *  - Asynchronous on `stream`; a wait inside the tensor-core kernel that
 *    runs out raises PC2_ST_TIMEOUT in the context's status word.
 *  - PC2_EINVAL: null pointers, even N, nsq < 0, unknown engine. */
int pc2_mont_sqr(pc2_ctx* ctx, const uint32_t* h_n, int limbs, const uint32_t* d_x, size_t count, int nsq, int engine,
                 uint32_t* d_y, pc2_stream_t stream);

/* ---- integer-multiplier throughput probe ---------------------------- *
 * A measurement aid (the paper has no counterpart): the modular
 * exponentiations of Eq. (itq1) and Sec. III-C are bound by the 32-bit
 * multiply pipe, and their roofline is quoted against the rate this probe
 * measures on the device.  kind:
 *   PC2_PROBE_LO    mad.lo.u32 (low half of a 32x32 product, plus an add)
 *   PC2_PROBE_HI    mad.hi.u32 (high half)
 *   PC2_PROBE_WIDE  mad.wide.u32 (a whole 32x32->64 product, plus a 64-bit add)
 *   PC2_PROBE_LOHI  a 32x32->64 product as mad.lo + mad.hi
 *   PC2_PROBE_DADD  add.rn.f64 (FP64 adds, the pipe of the z/v update)
 *   PC2_PROBE_ROW   the rows of a 64-limb Montgomery product as carry-flag
 *                   chains (mad.lo.cc / madc.hi.cc)
 *   PC2_PROBE_ROWW  the same rows as wide products with 64-bit adds, the
 *                   instruction pattern of the library's products
 * Launches blocks_per_sm x SMs CTAs of 128 threads (PC2_EINVAL when that
 * many cannot all be resident, or iters < 1); every thread runs `iters`
 * loop trips of independent accumulators.  Allocates its own small buffers
 * (cudaMalloc) and synchronises the stream.
 * Out (host): *ops = operations executed (multiplies of that kind; 32x32->64
 * products for WIDE, LOHI and ROW); *ms = CUDA-event time of the launch on
 * `stream`; *cycles = the longest CTA's clock64 cycles inside its loop;
 * *sms = the device's SM count (may be NULL). */
#define PC2_PROBE_LO 0
#define PC2_PROBE_HI 1
#define PC2_PROBE_WIDE 2
#define PC2_PROBE_LOHI 3
#define PC2_PROBE_ROW 4
#define PC2_PROBE_DADD 5
#define PC2_PROBE_ROWW 6
int pc2_probe_mul(int device, int kind, int blocks_per_sm, int iters, pc2_stream_t stream, double* ops, double* ms,
                  double* cycles, int* sms);

/* ---- decryption without device allocation ---------------------------- *
 * Not from the paper (it has no counterpart there): a variant of pc2_decrypt
 * for callers that may not allocate device memory -- a process held to a
 * fixed, pre-carved memory budget, a plugin that must not touch the device
 * allocator, or a latency path that cannot take the device-wide
 * synchronisation that cudaMalloc/cudaFree can imply.  It computes the same
 * result as pc2_decrypt (same arguments, no context) and calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *  - Scratch: a fixed array of PC2_NOALLOC_SCRATCH_BYTES compiled into the
 *    library, which every GPU that loads the library holds until the process
 *    exits.  The decryption's persistent grid is cut to the CTAs whose scratch
 *    fits, so it runs with fewer CTAs (lower throughput) than pc2_decrypt.
 *    Nothing in the array needs to start at zero: every word a call reads is
 *    written by that call first.
 *  - Runs on the calling thread's current device.  The FIRST call on each
 *    device looks up the array's device address (cudaGetSymbolAddress).
 *    With lazy module loading (the CUDA default) that lookup is also where
 *    the runtime loads this code's module and maps the 64 MiB array on the
 *    device, which can fail (PC2_ECUDA) or synchronise.  So make one warm-up
 *    call (count = 1 is enough) at start-up, before the caller's memory
 *    budget is carved and before any stream capture.
 *  - The address is cached per device for the life of the process: do not
 *    use this entry point across a cudaDeviceReset.
 *  - All calls share the one array: calls whose kernels overlap on a GPU
 *    (different streams, or different host threads) race and corrupt each
 *    other's results.  Order them on one stream.
 *  - Keys of 256 to 3072 bits; PC2_EUNSUPPORTED for 4096-bit keys.
 *  - PC2_ERANGE if one CTA's share of scratch for this key would exceed the
 *    array (it does not for the key sizes above); the element count itself
 *    is not limited.  The key's host-side constants are built and cached in
 *    host memory on its first decryption, as for pc2_decrypt.
 *  - PC2_EKEY for a public key; PC2_EINVAL for null pointers. */
#define PC2_NOALLOC_SCRATCH_BYTES (64u << 20)
int pc2_decrypt_noalloc(const pc2_key* key, const uint32_t* d_ct, size_t count, uint32_t* d_m, pc2_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* PC2_H */
