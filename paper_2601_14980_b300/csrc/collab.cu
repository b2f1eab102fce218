// collab.cu -- the collaborative CRT split of the paper's Sec. IV-C
// (Algorithm 3): edge node k computes the p^2 half of the master's
// encryptions and reduces its own ciphertexts mod p^2; the master computes
// the q^2 halves and recombines (Lemmas 1-2, Eq. (gA-C-B)).
//
// The paper leaves the obfuscation O(.) undefined; it is read as an
// additive mask: O(w) = w + kappa with kappa drawn by the master.  The edge
// reduces O(w) mod phi(p^2) (below 2 phi(p^2), so one conditional
// subtraction) and forms g^a r^n mod p^2 with g = n + 1, i.e. (1 + a n)
// (r^n mod p^2); the master multiplies that by g^(phi(p^2) - kappa mod
// phi(p^2)) = 1 + (phi(p^2) - kappa mod phi(p^2)) n mod p^2, which removes the
// mask, and recombines with its own half (1 + w n) (r^n mod q^2).  The
// result is the ciphertext E(w; r) of Eq. (itq1).  Both sides draw r from
// the same counter-based stream.
#include <cuda_runtime.h>

#include "../../include/pc2.h"
#include "ctx.hpp"
#include "keys.hpp"
#include "paillier_kernels.cuh"

namespace pc2 {
namespace {

template <int Lh>
struct Phi {
  uint32_t w[Lh];  // phi(p^2) = p (p - 1)
};

// v (Lh words, tiled input) minus phi when v >= phi, into column D.
template <int Lh>
__device__ __forceinline__ void reduce_phi(const Col& D, const uint32_t* v, size_t e, const Phi<Lh>& F) {
  for (int j = 0; j < Lh; ++j) D[j] = v[tiled_index(e, j, Lh)];
  if (g_ge(D, PArr{F.w}, Lh)) g_sub(D, D, PArr{F.w}, Lh);
}

// GM = 1 + a n (2 Lh words) for an a of Lh words in column Acol (a < n).
template <int Lh>
__device__ __forceinline__ void one_plus_an(const Col& GM, const Col& Acol, const uint32_t* n) {
  g_mul(GM, Acol, Lh, PArr{n}, Lh);
  uint64_t c = 1;
  for (int j = 0; j < 2 * Lh; ++j) {
    c += GM[j];
    GM[j] = (uint32_t)c;
    c >>= 32;
  }
}

template <int Lh>
__global__ void k_collab_mask(const uint64_t* __restrict__ w, const uint32_t* __restrict__ kappa, size_t count,
                              uint32_t* __restrict__ ow, int* status) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
    uint64_t c = w[e];
    for (int j = 0; j < Lh; ++j) {
      const uint64_t v = (uint64_t)kappa[tiled_index(e, j, Lh)] + (uint32_t)c;
      ow[tiled_index(e, j, Lh)] = (uint32_t)v;
      c = (c >> 32) + (v >> 32);
    }
    if (c) atomicOr(status, PC2_ST_RANGE);
  }
}

// Edge node: c'_masked = (1 + (O(w) mod phi(p^2)) n) (r^n mod p^2) mod p^2.
template <int Lh>
__global__ void __launch_bounds__(kThreads, min_blocks(Lh, 1))
    k_collab_edge_enc(const __grid_constant__ EncCrtParams<Lh> P, const Phi<Lh> F, const uint32_t* __restrict__ ow,
                      size_t count, uint32_t* __restrict__ cp, uint32_t* __restrict__ scratch, int tabw) {
  extern __shared__ uint32_t bsh_all[];
  const Grp<1> g;
  const Layout ly(1);
  const Col bsh{bsh_all + ly.gl, ly.G};
  const Col tab = ly.slot(scratch, 0);
  const int SW = 2 * Lh + 4;
  const Col X = ly.slot(scratch, tabw + 0 * SW), GM = ly.slot(scratch, tabw + 1 * SW),
            A = ly.slot(scratch, tabw + 2 * SW), B = ly.slot(scratch, tabw + 3 * SW),
            C = ly.slot(scratch, tabw + 4 * SW), TT = ly.slot(scratch, tabw + 5 * SW),
            OUT = ly.slot(scratch, tabw + 6 * SW), M = ly.slot(scratch, tabw + 7 * SW);
  for (size_t base = (size_t)blockIdx.x * ly.G; base < count; base += (size_t)ly.Gtot) {
    size_t e = base + ly.gl;
    const bool valid = e < count;
    if (!valid) e = count - 1;
    gen_r(X, P.seed, P.stream, P.e0 + e, Lh + 2, 2 * Lh);
    reduce_phi<Lh>(M, ow, e, F);
    one_plus_an<Lh>(GM, M, P.nwords);
    enc_half<Lh, 1>(P.mp, P.ep, P.lp, X, GM, OUT, A, B, C, TT, tab, bsh, g);
    if (valid)
      for (int j = 0; j < Lh; ++j) cp[tiled_index(e, j, Lh)] = OUT[j];
    __syncwarp();
  }
}

// Master: unmask the edge's half, its own half mod q^2, Eq. (gA-C-B).
template <int Lh>
__global__ void __launch_bounds__(kThreads, min_blocks(Lh, 1))
    k_collab_master_enc(const __grid_constant__ EncCrtParams<Lh> P, const Phi<Lh> F, const uint64_t* __restrict__ w,
                        const uint32_t* __restrict__ kappa, const uint32_t* __restrict__ cpm, size_t count,
                        uint32_t* __restrict__ out, uint32_t* __restrict__ scratch, int tabw, int* status) {
  extern __shared__ uint32_t bsh_all[];
  const Grp<1> g;
  const Layout ly(1);
  const Col bsh{bsh_all + ly.gl, ly.G};
  const Col tab = ly.slot(scratch, 0);
  const int SW = 2 * Lh + 4;
  const Col X = ly.slot(scratch, tabw + 0 * SW), GM = ly.slot(scratch, tabw + 1 * SW),
            A = ly.slot(scratch, tabw + 2 * SW), B = ly.slot(scratch, tabw + 3 * SW),
            C = ly.slot(scratch, tabw + 4 * SW), TT = ly.slot(scratch, tabw + 5 * SW),
            CP = ly.slot(scratch, tabw + 6 * SW), CQ = ly.slot(scratch, tabw + 7 * SW);
  for (size_t base = (size_t)blockIdx.x * ly.G; base < count; base += (size_t)ly.Gtot) {
    size_t e = base + ly.gl;
    const bool valid = e < count;
    if (!valid) e = count - 1;
    gen_r(X, P.seed, P.stream, P.e0 + e, Lh + 2, 2 * Lh);
    make_gm(GM, A, w, nullptr, e, P.nwords, Lh, 2 * Lh, valid, status);
    enc_half<Lh, 1>(P.mq, P.eq, P.lq, X, GM, CQ, A, B, C, TT, tab, bsh, g);
    // U = 1 + (phi - kappa mod phi) n mod p^2; c_p = c'_masked U mod p^2
    reduce_phi<Lh>(A, kappa, e, F);
    {
      uint64_t br = 0;  // A = phi - A
      for (int j = 0; j < Lh; ++j) {
        const uint64_t x = F.w[j], y = (uint64_t)A[j] + br;
        A[j] = (uint32_t)(x - y);
        br = x < y;
      }
    }
    one_plus_an<Lh>(GM, A, P.nwords);
    g_to_mont_2l(B, GM, P.mp.n, P.mp.r2, P.mp.r3, P.mp.np, Lh, C, CP, TT);  // U R mod p^2
    for (int j = 0; j < Lh; ++j) A[j] = cpm[tiled_index(e, j, Lh)];
    g_mont(CP, A, B, P.mp.n, P.mp.np, Lh, TT);                                // c_p
    // Eq. (gA-C-B): c = c_p + [(c_q - c_p) (p^2)^-1 mod q^2] p^2
    if (g_sub(A, CQ, CP, Lh)) g_add(A, A, PArr{P.mq.n}, Lh);
    g_copy_param(B, P.pinv2R, Lh);
    g_mont(C, A, B, P.mq.n, P.mq.np, Lh, TT);
    g_mul(X, C, Lh, PArr{P.p2}, Lh);
    uint64_t c = 0;
    for (int j = 0; j < 2 * Lh; ++j) {
      c += (uint64_t)X[j] + (j < Lh ? CP[j] : 0u);
      X[j] = (uint32_t)c;
      c >>= 32;
    }
    if (valid) write_tiled<1>(out, e, X, 2 * Lh, g);
    __syncwarp();
  }
}

// Edge node: x-hat' = x-hat mod p^2.
template <int Lh>
__global__ void __launch_bounds__(kThreads, min_blocks(Lh, 1))
    k_collab_edge_reduce(const __grid_constant__ DecParams<Lh> P, const uint32_t* __restrict__ ct, size_t count,
                         uint32_t* __restrict__ cp, uint32_t* __restrict__ scratch) {
  const Layout ly(1);
  const int SW = 2 * Lh + 4;
  const Col X = ly.slot(scratch, 0 * SW), A = ly.slot(scratch, 1 * SW), B = ly.slot(scratch, 2 * SW),
            C = ly.slot(scratch, 3 * SW), TT = ly.slot(scratch, 4 * SW);
  for (size_t base = (size_t)blockIdx.x * ly.G; base < count; base += (size_t)ly.Gtot) {
    size_t e = base + ly.gl;
    const bool valid = e < count;
    if (!valid) e = count - 1;
    for (int j = 0; j < 2 * Lh; ++j) X[j] = ct[tiled_index(e, j, 2 * Lh)];
    g_to_mont_2l(A, X, P.mp.n, P.mp.r2, P.mp.r3, P.mp.np, Lh, B, C, TT);  // x-hat R mod p^2
    g_zero(B, Lh);
    B[0] = 1u;
    g_mont(C, A, B, P.mp.n, P.mp.np, Lh, TT);                               // x-hat mod p^2
    if (valid)
      for (int j = 0; j < Lh; ++j) cp[tiled_index(e, j, Lh)] = C[j];
  }
}

// Master: m_p from the edge's residue, m_q from x-hat, Garner.
template <int Lh>
__global__ void __launch_bounds__(kThreads, min_blocks(Lh, 1))
    k_collab_master_dec(const __grid_constant__ DecParams<Lh> P, const uint32_t* __restrict__ ct,
                        const uint32_t* __restrict__ cpr, size_t count, uint32_t* __restrict__ out,
                        uint32_t* __restrict__ scratch, int tabw) {
  constexpr int Lp = Lh / 2;
  extern __shared__ uint32_t bsh_all[];
  const Grp<1> g;
  const Layout ly(1);
  const Col bsh{bsh_all + ly.gl, ly.G};
  const Col tab = ly.slot(scratch, 0);
  const int SW = 2 * Lh + 4;
  const Col X = ly.slot(scratch, tabw + 0 * SW), A = ly.slot(scratch, tabw + 1 * SW),
            B = ly.slot(scratch, tabw + 2 * SW), C = ly.slot(scratch, tabw + 3 * SW),
            TT = ly.slot(scratch, tabw + 4 * SW), MP = ly.slot(scratch, tabw + 5 * SW),
            MQ = ly.slot(scratch, tabw + 6 * SW);
  for (size_t base = (size_t)blockIdx.x * ly.G; base < count; base += (size_t)ly.Gtot) {
    size_t e = base + ly.gl;
    const bool valid = e < count;
    if (!valid) e = count - 1;
    for (int j = 0; j < 2 * Lh; ++j) X[j] = j < Lh ? cpr[tiled_index(e, j, Lh)] : 0u;
    dec_half<Lh, 1>(P.mp, P.ep, P.p, P.pnp, P.pinvlo, P.hpR, X, MP, A, B, C, TT, tab, bsh, g);
    for (int j = 0; j < 2 * Lh; ++j) X[j] = ct[tiled_index(e, j, 2 * Lh)];
    dec_half<Lh, 1>(P.mq, P.eq, P.q, P.qnp, P.qinvlo, P.hqR, X, MQ, A, B, C, TT, tab, bsh, g);
    if (g_sub(A, MQ, MP, Lp)) g_add(A, A, PArr{P.q}, Lp);
    g_copy_param(B, P.pinvqR, Lp);
    g_mont(C, A, B, P.q, P.qnp, Lp, TT);
    g_mul(X, C, Lp, PArr{P.p}, Lp);
    uint64_t c = 0;
    for (int j = 0; j < Lh; ++j) {
      c += (uint64_t)X[j] + (j < Lp ? MP[j] : 0u);
      X[j] = (uint32_t)c;
      c >>= 32;
    }
    if (valid) write_tiled<1>(out, e, X, Lh, g);
    __syncwarp();
  }
}

// ------------------------------------------------------------------ host side
template <class K>
int persistent_grid(K kern, size_t smem, int sms) {
  int per = 0;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kThreads, smem) != cudaSuccess || per < 1) return -1;
  return per * sms;
}

template <int Lh>
Phi<Lh> phi_of(const pc2_key* key) {
  Phi<Lh> F;
  mul(key->p, sub(key->p, Big(1))).to_words(F.w, Lh);
  return F;
}

size_t group_words(int tabw, int cols, int Lh) { return (size_t)tabw + (size_t)cols * (2 * Lh + 4); }

template <int Lh>
int edge_encrypt(pc2_ctx* ctx, const pc2_key* key, const uint32_t* ow, size_t count, uint64_t seed, uint32_t stream,
                 uint64_t e0, uint32_t* cp, cudaStream_t st) {
  int rc = PC2_OK;
  auto P0 = enc_params<Lh>(key, &rc);
  if (!P0) return rc;
  std::unique_ptr<EncCrtParams<Lh>> P(new (std::nothrow) EncCrtParams<Lh>(*P0));
  if (!P) return PC2_ENOMEM;
  P->seed = seed;
  P->stream = stream;
  P->e0 = e0;
  const size_t smem = (size_t)Lh * kThreads * 4;
  auto kern = k_collab_edge_enc<Lh>;
  const int grid = persistent_grid(kern, smem, ctx->sms);
  if (grid < 0) return PC2_ECUDA;
  const int w = P->ep.w > P->eq.w ? P->ep.w : P->eq.w;
  const int tabw = (1 << (w - 1)) * Lh;
  uint32_t* scratch = ctx_scratch_get(ctx, group_words(tabw, 8, Lh) * (size_t)grid * kThreads * 4);
  if (!scratch) return PC2_ENOMEM;
  kern<<<grid, kThreads, smem, st>>>(*P, phi_of<Lh>(key), ow, count, cp, scratch, tabw);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

template <int Lh>
int master_encrypt(pc2_ctx* ctx, const pc2_key* key, const uint64_t* w, const uint32_t* kappa, const uint32_t* cpm,
                   size_t count, uint64_t seed, uint32_t stream, uint64_t e0, uint32_t* out, cudaStream_t st) {
  int rc = PC2_OK;
  auto P0 = enc_params<Lh>(key, &rc);
  if (!P0) return rc;
  std::unique_ptr<EncCrtParams<Lh>> P(new (std::nothrow) EncCrtParams<Lh>(*P0));
  if (!P) return PC2_ENOMEM;
  P->seed = seed;
  P->stream = stream;
  P->e0 = e0;
  P->mwords = 2;
  const size_t smem = (size_t)Lh * kThreads * 4;
  auto kern = k_collab_master_enc<Lh>;
  const int grid = persistent_grid(kern, smem, ctx->sms);
  if (grid < 0) return PC2_ECUDA;
  const int wd = P->ep.w > P->eq.w ? P->ep.w : P->eq.w;
  const int tabw = (1 << (wd - 1)) * Lh;
  uint32_t* scratch = ctx_scratch_get(ctx, group_words(tabw, 8, Lh) * (size_t)grid * kThreads * 4);
  if (!scratch) return PC2_ENOMEM;
  kern<<<grid, kThreads, smem, st>>>(*P, phi_of<Lh>(key), w, kappa, cpm, count, out, scratch, tabw, ctx->status);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

template <int Lh>
int edge_reduce(pc2_ctx* ctx, const pc2_key* key, const uint32_t* ct, size_t count, uint32_t* cp, cudaStream_t st) {
  int rc = PC2_OK;
  auto P = dec_params<Lh>(key, &rc);
  if (!P) return rc;
  auto kern = k_collab_edge_reduce<Lh>;
  const int grid = persistent_grid(kern, 0, ctx->sms);
  if (grid < 0) return PC2_ECUDA;
  uint32_t* scratch = ctx_scratch_get(ctx, group_words(0, 5, Lh) * (size_t)grid * kThreads * 4);
  if (!scratch) return PC2_ENOMEM;
  kern<<<grid, kThreads, 0, st>>>(*P, ct, count, cp, scratch);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

template <int Lh>
int master_decrypt(pc2_ctx* ctx, const pc2_key* key, const uint32_t* ct, const uint32_t* cp, size_t count,
                   uint32_t* out, cudaStream_t st) {
  int rc = PC2_OK;
  auto P = dec_params<Lh>(key, &rc);
  if (!P) return rc;
  const size_t smem = (size_t)Lh * kThreads * 4;
  auto kern = k_collab_master_dec<Lh>;
  const int grid = persistent_grid(kern, smem, ctx->sms);
  if (grid < 0) return PC2_ECUDA;
  const int w = P->ep.w > P->eq.w ? P->ep.w : P->eq.w;
  const int tabw = (1 << (w - 1)) * Lh;
  uint32_t* scratch = ctx_scratch_get(ctx, group_words(tabw, 7, Lh) * (size_t)grid * kThreads * 4);
  if (!scratch) return PC2_ENOMEM;
  kern<<<grid, kThreads, smem, st>>>(*P, ct, cp, count, out, scratch, tabw);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

}  // namespace
}  // namespace pc2

using namespace pc2;

#define PC2_COLLAB_DISPATCH(Lh, call) \
  switch (Lh) {                       \
    case 8: return call(8);           \
    case 16: return call(16);         \
    case 32: return call(32);         \
    case 64: return call(64);         \
    default: return PC2_EUNSUPPORTED; \
  }

static int collab_check(pc2_ctx* ctx, const pc2_key* key) {
  if (!ctx || !key) return PC2_EINVAL;
  if (!key->priv) return PC2_EKEY;
  return PC2_OK;
}

extern "C" int pc2_collab_mask(pc2_ctx* ctx, const pc2_key* key, const uint64_t* d_w, const uint32_t* d_kappa,
                               size_t count, uint32_t* d_ow, pc2_stream_t stream) {
  if (!ctx || !key) return PC2_EINVAL;
  if (!count) return PC2_OK;
  if (!d_w || !d_kappa || !d_ow) return PC2_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  const size_t blocks = (count + 255) / 256;
  const unsigned grid = (unsigned)(blocks < (size_t)ctx->sms * 8 ? blocks : (size_t)ctx->sms * 8);
#define PC2_MASK(L) (k_collab_mask<L><<<grid, 256, 0, st>>>(d_w, d_kappa, count, d_ow, ctx->status), \
                     cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA)
  PC2_COLLAB_DISPATCH(key->Lh, PC2_MASK)
#undef PC2_MASK
}

extern "C" int pc2_collab_edge_encrypt(pc2_ctx* ctx, const pc2_key* key, const uint32_t* d_ow, size_t count,
                                       uint64_t seed, uint32_t stream, uint64_t e0, uint32_t* d_cp,
                                       pc2_stream_t cstream) {
  int rc = collab_check(ctx, key);
  if (rc != PC2_OK) return rc;
  if (!count) return PC2_OK;
  if (!d_ow || !d_cp) return PC2_EINVAL;
  const cudaStream_t st = (cudaStream_t)cstream;
#define PC2_EDGE_ENC(L) edge_encrypt<L>(ctx, key, d_ow, count, seed, stream, e0, d_cp, st)
  PC2_COLLAB_DISPATCH(key->Lh, PC2_EDGE_ENC)
#undef PC2_EDGE_ENC
}

extern "C" int pc2_collab_master_encrypt(pc2_ctx* ctx, const pc2_key* key, const uint64_t* d_w,
                                         const uint32_t* d_kappa, const uint32_t* d_cp, size_t count, uint64_t seed,
                                         uint32_t stream, uint64_t e0, uint32_t* d_ct, pc2_stream_t cstream) {
  int rc = collab_check(ctx, key);
  if (rc != PC2_OK) return rc;
  if (!count) return PC2_OK;
  if (!d_w || !d_kappa || !d_cp || !d_ct) return PC2_EINVAL;
  const cudaStream_t st = (cudaStream_t)cstream;
#define PC2_MASTER_ENC(L) master_encrypt<L>(ctx, key, d_w, d_kappa, d_cp, count, seed, stream, e0, d_ct, st)
  PC2_COLLAB_DISPATCH(key->Lh, PC2_MASTER_ENC)
#undef PC2_MASTER_ENC
}

extern "C" int pc2_collab_edge_reduce(pc2_ctx* ctx, const pc2_key* key, const uint32_t* d_ct, size_t count,
                                      uint32_t* d_cp, pc2_stream_t cstream) {
  int rc = collab_check(ctx, key);
  if (rc != PC2_OK) return rc;
  if (!count) return PC2_OK;
  if (!d_ct || !d_cp) return PC2_EINVAL;
  const cudaStream_t st = (cudaStream_t)cstream;
#define PC2_EDGE_RED(L) edge_reduce<L>(ctx, key, d_ct, count, d_cp, st)
  PC2_COLLAB_DISPATCH(key->Lh, PC2_EDGE_RED)
#undef PC2_EDGE_RED
}

extern "C" int pc2_collab_master_decrypt(pc2_ctx* ctx, const pc2_key* key, const uint32_t* d_ct,
                                         const uint32_t* d_cp, size_t count, uint32_t* d_m, pc2_stream_t cstream) {
  int rc = collab_check(ctx, key);
  if (rc != PC2_OK) return rc;
  if (!count) return PC2_OK;
  if (!d_ct || !d_cp || !d_m) return PC2_EINVAL;
  const cudaStream_t st = (cudaStream_t)cstream;
#define PC2_MASTER_DEC(L) master_decrypt<L>(ctx, key, d_ct, d_cp, count, d_m, st)
  PC2_COLLAB_DISPATCH(key->Lh, PC2_MASTER_DEC)
#undef PC2_MASTER_DEC
}
