// admm.cpp -- the 3P-ADMM-PC2 loop on one GPU (Algorithm 1 of the paper).
//
// The K edge nodes are simulated as segments of device vectors.  One round:
//   master   Gamma2(z), Gamma2(-v) and their per-node sums      (k_admm_quant)
//            z-hat = E(Gamma2(z)), (-v)-hat = E(Gamma2(-v))     (Eq. (uyt12), CRT path)
//   edge k   s-hat = z-hat (+) (-v)-hat                         (Definition 1)
//            x-hat_k = alpha-hat_k (+) Gamma2(Bbar_k) (x) s-hat  (Eq. (itq2), k_matvec)
//   master   D = decrypt(x-hat), x = exact decode of D,
//            z = S_kappa(v + x), v = v + x - z                   (k_admm_update)
// The batched path runs every node in the same launches and replays the
// round as one CUDA graph (the r-stream id comes from a device round
// counter); the per-node path launches each node separately.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "../../include/pc2.h"
#include "ctx.hpp"
#include "keys.hpp"
#include "pc2_admm.h"
#include "pc2_kernels.h"

namespace {

template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  int alloc(size_t count) {
    n = count;
    if (!count) return PC2_OK;
    return cudaMalloc(&p, count * sizeof(T)) == cudaSuccess ? PC2_OK : PC2_ENOMEM;
  }
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

}  // namespace

struct pc2_admm {
  pc2_ctx* ctx = nullptr;
  const pc2_key* key = nullptr;
  int K = 0, N = 0, Lh = 0, L2 = 0;
  double lambda = 0, rho = 0, zmin = 0, zmax = 0, kappa = 0;
  int log2s = 0;
  long long mS = 0, S = 0;
  double scale = 0, qmax = 0, inv_s2 = 0;
  uint64_t seed = 0;
  int per_node = 0;
  int c = 4, nwin = 1;
  std::vector<int> off, tile_start;
  std::vector<long long> boffh;
  int ntiles = 0;
  int mv_T = 1;  // lanes per row of the matvec (fixed at creation: it sets the row tiles)
  int mv_mode = 0;  // matvec form: 0 automatic, 1 rows per CTA, 2 windows spread over CTAs
  DevBuf<uint32_t> part;  // window-parallel partial products (nwin x N, tiled)
  DevBuf<double> alpha, Bbar, x, z, v;
  DevBuf<uint32_t> bq, alpha_hat, shat, smont, xhat, D, round_ctr, bitlen;
  DevBuf<uint32_t> zvhat;  // z-hat (elements [0, N)) then (-v)-hat (from element Npad) in one tiled array
  uint32_t* zhat = nullptr;
  uint32_t* vhat = nullptr;
  DevBuf<long long> boff, brow;
  DevBuf<int> node_of, node_off, node_size, tile_node, tile_row0;
  DevBuf<uint64_t> zv, tmp64;  // Gamma2(z) then Gamma2(-v), adjacent (one encryption launch)
  uint64_t* zq = nullptr;
  uint64_t* vq = nullptr;
  int Npad = 0;                 // N rounded up to a whole tile
  DevBuf<unsigned long long> asum;
  std::shared_ptr<void> mvp, modp;  // cached MatvecParams<L2> / ModConst<L2> of n^2
  cudaGraphExec_t graph = nullptr;
  cudaStream_t cap = nullptr;
  std::vector<uint8_t> present;  // per node: its segment of the next round has arrived (1 by default)
  ~pc2_admm() {
    if (graph) cudaGraphExecDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
  }
  size_t ctw() const { return pc2_tiled_words((size_t)N, L2); }
};

namespace pc2 {

template <int L2, int T>
static int matvec_launch_t(pc2_admm* A, int tile0, int ntl, cudaStream_t st) {
  if (!A->mvp) {
    std::shared_ptr<MatvecParams<L2>> p(new (std::nothrow) MatvecParams<L2>);
    if (!p) return PC2_ENOMEM;
    std::memset(p.get(), 0, sizeof(MatvecParams<L2>));
    fill_mod(p->m, A->key->n2);
    p->c = A->c;
    p->nwin = A->nwin;
    A->mvp = p;
  }
  MatvecParams<L2> P = *std::static_pointer_cast<MatvecParams<L2>>(A->mvp);
  P.ntiles = ntl;
  // few row tiles: spread the bucket windows of each row over CTAs too
  const int cap = matvec_win_grid<L2, T>(1 << 30, A->ctx->sms);
  if (cap < 1) return PC2_ECUDA;
  const bool win_par = A->nwin > 1 && (A->mv_mode == 2 || (A->mv_mode == 0 && 2 * ntl < cap));
  if (win_par) {
    const int grid = std::min(ntl * A->nwin, cap);
    uint32_t* scr = ctx_scratch_get(A->ctx, matvec_scratch_words<L2, T>(A->c, grid) * 4);
    if (!scr) return PC2_ENOMEM;
    if (!A->part.p && A->part.alloc(pc2_tiled_words((size_t)A->N * A->nwin, L2))) return PC2_ENOMEM;
    return launch_matvec_win<L2, T>(P, A->alpha_hat.p, A->smont.p, A->bq.p, A->boff.p, A->node_off.p,
                                    A->tile_node.p + tile0, A->tile_row0.p + tile0, A->N, A->part.p, A->xhat.p, scr,
                                    grid, A->ctx->sms, st);
  }
  const int grid = matvec_grid<L2, T>(ntl, A->ctx->sms);
  if (grid < 1) return PC2_ECUDA;
  uint32_t* scr = ctx_scratch_get(A->ctx, matvec_scratch_words<L2, T>(A->c, grid) * 4);
  if (!scr) return PC2_ENOMEM;
  return launch_matvec<L2, T>(P, A->alpha_hat.p, A->smont.p, A->bq.p, A->boff.p, A->node_off.p, A->tile_node.p + tile0,
                              A->tile_row0.p + tile0, A->xhat.p, scr, grid, st);
}

// Lanes per row of the matvec: the count picked at creation (built sets:
// 1, 2, 4 for 16 limbs; 1, 2, 4, 8 for 32 and 64; 4, 8 for 128, 192 and 256).
template <int L2>
static int matvec_launch(pc2_admm* A, int tile0, int ntl, cudaStream_t st) {
  switch (A->mv_T) {
    case 1: if constexpr (L2 <= 64) return matvec_launch_t<L2, 1>(A, tile0, ntl, st); break;
    case 2: if constexpr (L2 <= 64) return matvec_launch_t<L2, 2>(A, tile0, ntl, st); break;
    case 4: return matvec_launch_t<L2, 4>(A, tile0, ntl, st);
    case 8: if constexpr (L2 >= 32) return matvec_launch_t<L2, 8>(A, tile0, ntl, st); break;
  }
  return PC2_EUNSUPPORTED;
}

template <int L2>
static int to_mont_launch(pc2_admm* A, cudaStream_t st) {
  if (!A->modp) {
    std::shared_ptr<ModConst<L2>> p(new (std::nothrow) ModConst<L2>);
    if (!p) return PC2_ENOMEM;
    fill_mod(*p, A->key->n2);
    A->modp = p;
  }
  return launch_to_mont_rows<L2, lanes_for(L2)>(*std::static_pointer_cast<ModConst<L2>>(A->modp), A->shat.p, A->N,
                                                A->smont.p, A->ctx->sms, st);
}

static int dispatch_matvec(pc2_admm* A, int tile0, int ntl, cudaStream_t st) {
  switch (A->L2) {
    case 16: return matvec_launch<16>(A, tile0, ntl, st);
    case 32: return matvec_launch<32>(A, tile0, ntl, st);
    case 64: return matvec_launch<64>(A, tile0, ntl, st);
    case 128: return matvec_launch<128>(A, tile0, ntl, st);
    case 192: return matvec_launch<192>(A, tile0, ntl, st);
    case 256: return matvec_launch<256>(A, tile0, ntl, st);
    default: return PC2_EUNSUPPORTED;
  }
}
static int dispatch_to_mont(pc2_admm* A, cudaStream_t st) {
  switch (A->L2) {
    case 16: return to_mont_launch<16>(A, st);
    case 32: return to_mont_launch<32>(A, st);
    case 64: return to_mont_launch<64>(A, st);
    case 128: return to_mont_launch<128>(A, st);
    case 192: return to_mont_launch<192>(A, st);
    case 256: return to_mont_launch<256>(A, st);
    default: return PC2_EUNSUPPORTED;
  }
}

// Eq. (itq2) on one n x n block outside an ADMM object: K_ij < 2^kbits, scratch
// from the context (Montgomery form of s, tile tables, window products, kernel
// scratch), same kernels and choices as the round's matvec.
template <int L2, int T>
static int block_matvec(pc2_ctx* ctx, const pc2_key* key, const uint32_t* alpha, const uint32_t* s, const uint32_t* K,
                        int n, int kbits, uint32_t* out, cudaStream_t st) {
  const int G = kThreads / T, ntiles = (n + G - 1) / G;
  // bucket window: fewest products per row, nwin * (n + 2 (2^c - 1) + c + 1)
  int c = 1, nwin = kbits;
  double best = 1e300;
  for (int cc = 1; cc <= 8; ++cc) {
    const int nw = (kbits + cc - 1) / cc;
    const double cost = (double)nw * (n + 2.0 * ((1 << cc) - 1) + cc + 1);
    if (cost < best) {
      best = cost;
      c = cc;
      nwin = nw;
    }
  }
  std::unique_ptr<MatvecParams<L2>> P(new (std::nothrow) MatvecParams<L2>);
  std::unique_ptr<ModConst<L2>> M(new (std::nothrow) ModConst<L2>);
  if (!P || !M) return PC2_ENOMEM;
  std::memset(P.get(), 0, sizeof(MatvecParams<L2>));
  fill_mod(*M, key->n2);
  P->m = *M;
  P->c = c;
  P->nwin = nwin;
  P->ntiles = ntiles;
  const int cap = matvec_win_grid<L2, T>(1 << 30, ctx->sms);
  if (cap < 1) return PC2_ECUDA;
  const bool win_par = nwin > 1 && 2 * ntiles < cap;
  const int grid = win_par ? std::min(ntiles * nwin, cap) : matvec_grid<L2, T>(ntiles, ctx->sms);
  if (grid < 1) return PC2_ECUDA;
  // scratch layout (words, 64-word aligned): smont | tables | window products | kernel scratch
  auto up = [](size_t w) { return (w + 63) / 64 * 64; };
  const size_t w_smont = up((size_t)n * L2), w_tab = up(4 + 2 * (size_t)ntiles + 2);
  const size_t w_part = win_par ? up(pc2_tiled_words((size_t)n * nwin, L2)) : 0;
  const size_t w_kern = matvec_scratch_words<L2, T>(c, grid);
  uint32_t* base = ctx_scratch_get(ctx, (w_smont + w_tab + w_part + w_kern) * 4);
  if (!base) return PC2_ENOMEM;
  uint32_t* smont = base;
  uint32_t* tab = base + w_smont;
  uint32_t* part = tab + w_tab;
  uint32_t* kscr = part + w_part;
  // tables: node_off {0, n}, boff {0} (64-bit), tile_node, tile_row0
  std::vector<int> ht(w_tab, 0);
  ht[0] = 0;
  ht[1] = n;
  long long* boff_h = reinterpret_cast<long long*>(&ht[2]);
  *boff_h = 0;
  for (int t = 0; t < ntiles; ++t) {
    ht[4 + t] = 0;
    ht[4 + ntiles + t] = t * G;
  }
  if (cudaMemcpyAsync(tab, ht.data(), w_tab * 4, cudaMemcpyHostToDevice, st) != cudaSuccess) return PC2_ECUDA;
  const int* node_off = reinterpret_cast<const int*>(tab);
  const long long* boff = reinterpret_cast<const long long*>(tab + 2);
  const int* tile_node = reinterpret_cast<const int*>(tab + 4);
  const int* tile_row0 = reinterpret_cast<const int*>(tab + 4 + ntiles);
  int rc = launch_to_mont_rows<L2, lanes_for(L2)>(*M, s, n, smont, ctx->sms, st);
  if (rc) return rc;
  if (win_par)
    return launch_matvec_win<L2, T>(*P, alpha, smont, K, boff, node_off, tile_node, tile_row0, n, part, out, kscr,
                                    grid, ctx->sms, st);
  return launch_matvec<L2, T>(*P, alpha, smont, K, boff, node_off, tile_node, tile_row0, out, kscr, grid, st);
}

template <int L2>
static int block_matvec_any(pc2_ctx* ctx, const pc2_key* key, const uint32_t* alpha, const uint32_t* s,
                            const uint32_t* K, int n, int kbits, uint32_t* out, cudaStream_t st) {
  switch (pick_config(ctx, OP_MATVEC, L2, (size_t)n).T) {
    case 1: if constexpr (L2 <= 64) return block_matvec<L2, 1>(ctx, key, alpha, s, K, n, kbits, out, st); break;
    case 2: if constexpr (L2 <= 64) return block_matvec<L2, 2>(ctx, key, alpha, s, K, n, kbits, out, st); break;
    case 4: return block_matvec<L2, 4>(ctx, key, alpha, s, K, n, kbits, out, st);
    case 8: if constexpr (L2 >= 32) return block_matvec<L2, 8>(ctx, key, alpha, s, K, n, kbits, out, st); break;
  }
  return PC2_EUNSUPPORTED;
}

#define PC2_TRY(x)            \
  do {                        \
    const int rc_ = (x);      \
    if (rc_ != PC2_OK) return rc_; \
  } while (0)

// One private round, all nodes batched.
static int round_batched(pc2_admm* A, cudaStream_t st) {
  pc2_ctx* ctx = A->ctx;
  if (cudaMemsetAsync(A->asum.p, 0, A->K * sizeof(unsigned long long), st) != cudaSuccess) return PC2_ECUDA;
  PC2_TRY(launch_admm_quant(A->z.p, A->v.p, A->N, A->node_of.p, A->zmin, A->scale, A->qmax, A->zq, A->vq,
                            A->asum.p, ctx->status, ctx->sms, st));
  // z-hat and (-v)-hat in one call: elements [0, N) are Gamma2(z) (r-stream kind 1),
  // [N, 2N) are Gamma2(-v) (kind 2, counter restarting at 0, tiled from element Npad)
  PC2_TRY(encrypt_round(ctx, A->key, A->zq, 2 * (size_t)A->N, A->seed, A->round_ctr.p, 1, 0, A->zvhat.p, st, 0,
                        (size_t)A->N, 2, (size_t)A->Npad));
  PC2_TRY(pc2_hom_add(ctx, A->key, A->zhat, A->vhat, A->N, A->shat.p, (pc2_stream_t)st));
  PC2_TRY(dispatch_to_mont(A, st));
  PC2_TRY(dispatch_matvec(A, 0, A->ntiles, st));
  PC2_TRY(pc2_decrypt(ctx, A->key, A->xhat.p, A->N, A->D.p, (pc2_stream_t)st));
  return launch_admm_update(A->D.p, A->Lh, A->N, A->node_of.p, A->node_size.p, A->brow.p, A->asum.p, A->mS, A->S,
                            A->inv_s2, A->kappa, A->x.p, A->z.p, A->v.p, ctx->status, A->round_ctr.p, ctx->sms, st);
}

}  // namespace pc2

using namespace pc2;

extern "C" {

int pc2_quantize(pc2_ctx* ctx, const double* d_u, size_t n, double zmin, double zmax, int log2_scale, int gamma,
                 int negate, uint64_t* d_q, pc2_stream_t stream) {
  if (!ctx || (n && (!d_u || !d_q)) || (gamma != 1 && gamma != 2) || log2_scale < 0 || log2_scale > 40 ||
      !(zmax > zmin))
    return PC2_EINVAL;
  if (!n) return PC2_OK;
  const double S = std::ldexp(1.0, log2_scale);
  const double delta = std::rint((zmax - zmin) * S);
  const double scale = gamma == 1 ? S * S : S;
  const double qmax = gamma == 1 ? delta * S : delta;
  if (qmax >= 18446744073709551616.0) return PC2_ERANGE;
  return launch_quantize(d_u, n, zmin, scale, qmax, negate, d_q, ctx->status, nullptr, ctx->sms, (cudaStream_t)stream);
}

int pc2_admm_create(pc2_ctx* ctx, const pc2_key* key, const pc2_admm_params* prm, const double* d_alpha,
                    const double* d_Bbar, pc2_admm** out, pc2_stream_t stream) {
  if (!ctx || !key || !prm || !d_alpha || !d_Bbar || !out || prm->nodes <= 0 || !prm->node_sizes) return PC2_EINVAL;
  if (!key->priv) return PC2_EKEY;
  *out = nullptr;
  const cudaStream_t st = (cudaStream_t)stream;
  std::unique_ptr<pc2_admm> A(new (std::nothrow) pc2_admm);
  if (!A) return PC2_ENOMEM;
  A->ctx = ctx;
  A->key = key;
  A->K = prm->nodes;
  A->Lh = key->Lh;
  A->L2 = 2 * key->Lh;
  A->lambda = prm->lambda;
  A->rho = prm->rho;
  A->zmin = prm->zmin;
  A->zmax = prm->zmax;
  A->log2s = prm->log2_scale;
  A->seed = prm->seed;
  A->per_node = prm->per_node;
  if (!(prm->rho > 0) || !(prm->lambda >= 0) || !(prm->zmax > prm->zmin) || prm->log2_scale < 1 ||
      prm->log2_scale > 30)
    return PC2_EINVAL;
  A->kappa = prm->lambda / prm->rho;
  A->S = 1LL << prm->log2_scale;
  A->scale = (double)A->S;
  const double ms = prm->zmin * A->scale;
  if (ms != std::floor(ms) || std::fabs(ms) > 9.0e15) return PC2_EINVAL;  // zmin * S must be an integer
  A->mS = (long long)ms;
  A->qmax = std::rint((prm->zmax - prm->zmin) * A->scale);
  A->inv_s2 = std::ldexp(1.0, -2 * prm->log2_scale);
  // node layout and CTA row tiles (a tile never straddles two nodes)
  size_t Ntot = 0;
  for (int k = 0; k < A->K; ++k) Ntot += prm->node_sizes[k] > 0 ? (size_t)prm->node_sizes[k] : 0;
  A->mv_T = pick_config(ctx, OP_MATVEC, A->L2, Ntot).T;
  const int G = kThreads / A->mv_T;
  A->off.assign(A->K + 1, 0);
  A->boffh.assign(A->K, 0);
  std::vector<int> nof, tnode, trow;
  long long bsum = 0;
  for (int k = 0; k < A->K; ++k) {
    const int nk = prm->node_sizes[k];
    if (nk <= 0) return PC2_EINVAL;
    A->off[k + 1] = A->off[k] + nk;
    A->boffh[k] = bsum;
    bsum += (long long)nk * nk;
    A->tile_start.push_back((int)tnode.size());
    for (int r = 0; r < nk; r += G) {
      tnode.push_back(k);
      trow.push_back(A->off[k] + r);
    }
    for (int r = 0; r < nk; ++r) nof.push_back(k);
  }
  A->tile_start.push_back((int)tnode.size());
  A->N = A->off[A->K];
  A->Npad = (A->N + 31) / 32 * 32;
  A->ntiles = (int)tnode.size();
  const int N = A->N;
  std::vector<int> nsz(A->K);
  for (int k = 0; k < A->K; ++k) nsz[k] = prm->node_sizes[k];
  const size_t ctw = A->ctw();
  if (A->alpha.alloc(N) || A->Bbar.alloc(bsum) || A->x.alloc(N) || A->z.alloc(N) || A->v.alloc(N) ||
      A->bq.alloc(bsum) || A->alpha_hat.alloc(ctw) || A->zvhat.alloc(2 * pc2_tiled_words(A->Npad, A->L2)) ||
      A->shat.alloc(ctw) || A->smont.alloc((size_t)N * A->L2) || A->xhat.alloc(ctw) ||
      A->D.alloc(pc2_tiled_words(N, A->Lh)) || A->round_ctr.alloc(1) || A->bitlen.alloc(1) || A->boff.alloc(A->K) ||
      A->brow.alloc(N) || A->node_of.alloc(N) || A->node_off.alloc(A->K + 1) || A->node_size.alloc(A->K) ||
      A->tile_node.alloc(A->ntiles) || A->tile_row0.alloc(A->ntiles) || A->zv.alloc(2 * (size_t)N) ||
      A->tmp64.alloc(bsum > N ? bsum : N) || A->asum.alloc(A->K))
    return PC2_ENOMEM;
  A->zq = A->zv.p;
  A->vq = A->zv.p + N;
  A->zhat = A->zvhat.p;
  A->vhat = A->zvhat.p + pc2_tiled_words(A->Npad, A->L2);
  auto h2d = [&](void* d, const void* h, size_t bytes) {
    return cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, st) == cudaSuccess;
  };
  if (!h2d(A->node_of.p, nof.data(), N * 4) || !h2d(A->node_off.p, A->off.data(), (A->K + 1) * 4) ||
      !h2d(A->node_size.p, nsz.data(), A->K * 4) || !h2d(A->boff.p, A->boffh.data(), A->K * 8) ||
      !h2d(A->tile_node.p, tnode.data(), A->ntiles * 4) || !h2d(A->tile_row0.p, trow.data(), A->ntiles * 4))
    return PC2_ECUDA;
  if (cudaMemcpyAsync(A->alpha.p, d_alpha, N * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(A->Bbar.p, d_Bbar, bsum * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(A->bitlen.p, 0, 4, st) != cudaSuccess)
    return PC2_ECUDA;
  // Gamma2(Bbar_k) as 32-bit digits, their widest bit length, row sums
  PC2_TRY(launch_quantize(A->Bbar.p, bsum, A->zmin, A->scale, A->qmax, 0, A->tmp64.p, ctx->status, A->bitlen.p,
                          ctx->sms, st));
  PC2_TRY(launch_narrow(A->tmp64.p, bsum, A->bq.p, ctx->status, ctx->sms, st));
  PC2_TRY(launch_rowsum(A->bq.p, A->boff.p, A->node_of.p, A->node_off.p, N, A->brow.p, ctx->sms, st));
  // alpha-hat = E(Gamma1(alpha)), r-stream 0 (round 0, kind 0)
  PC2_TRY(launch_quantize(A->alpha.p, N, A->zmin, A->scale * A->scale, A->qmax * A->scale, 0, A->tmp64.p,
                          ctx->status, nullptr, ctx->sms, st));
  PC2_TRY(pc2_encrypt(ctx, key, A->tmp64.p, N, A->seed, 0, 0, A->alpha_hat.p, stream));
  uint32_t bits_or = 0;
  if (cudaMemcpyAsync(&bits_or, A->bitlen.p, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PC2_ECUDA;
  int bits = 0;
  while (bits < 32 && (bits_or >> bits)) ++bits;
  if (bits == 0) bits = 1;
  // bucket window: fewest products per row, nwin * (N_k + 2 (2^c - 1) + c + 1)
  int maxnk = 0;
  for (int k = 0; k < A->K; ++k) maxnk = nsz[k] > maxnk ? nsz[k] : maxnk;
  double best = 1e300;
  for (int c = 1; c <= 8; ++c) {
    const int nw = (bits + c - 1) / c;
    const double cost = (double)nw * (maxnk + 2.0 * ((1 << c) - 1) + c + 1);
    if (cost < best) { best = cost; A->c = c; A->nwin = nw; }
  }
  *out = A.release();
  return pc2_admm_reset(*out, stream);
}

int pc2_admm_reset(pc2_admm* A, pc2_stream_t stream) {
  if (!A) return PC2_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  const uint32_t one = 1;
  if (cudaMemsetAsync(A->x.p, 0, A->N * 8, st) != cudaSuccess || cudaMemsetAsync(A->z.p, 0, A->N * 8, st) ||
      cudaMemsetAsync(A->v.p, 0, A->N * 8, st) ||
      cudaMemcpyAsync(A->round_ctr.p, &one, 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PC2_ECUDA;
  return PC2_OK;
}

void pc2_admm_destroy(pc2_admm* A) {
  if (!A) return;
  cudaSetDevice(A->ctx->device);
  cudaDeviceSynchronize();
  delete A;
}

int pc2_admm_set_node_present(pc2_admm* A, int node, int present) {
  if (!A || node < 0 || node >= A->K) return PC2_EINVAL;
  if ((int)A->present.size() != A->K) A->present.assign(A->K, 1);
  A->present[node] = present ? 1 : 0;
  return PC2_OK;
}

int pc2_admm_round(pc2_admm* A, int rounds, pc2_stream_t stream) {
  if (!A || rounds < 0) return PC2_EINVAL;
  // a round needs every edge node's segment: report a missing one before
  // any launch, with the state untouched, so the caller can retry
  for (const uint8_t p : A->present)
    if (!p) return PC2_EMISSING;
  const cudaStream_t st = (cudaStream_t)stream;
  pc2_ctx* ctx = A->ctx;
  for (int r = 0; r < rounds; ++r) {
    if (A->per_node) {
      // every node launched on its own (the plain per-node path)
      if (cudaMemsetAsync(A->asum.p, 0, A->K * sizeof(unsigned long long), st) != cudaSuccess) return PC2_ECUDA;
      PC2_TRY(launch_admm_quant(A->z.p, A->v.p, A->N, A->node_of.p, A->zmin, A->scale, A->qmax, A->zq, A->vq,
                                A->asum.p, ctx->status, ctx->sms, st));
      for (int k = 0; k < A->K; ++k) {
        const int o = A->off[k], nk = A->off[k + 1] - o;
        PC2_TRY(encrypt_round(ctx, A->key, A->zq + o, nk, A->seed, A->round_ctr.p, 1, o, A->zhat, st, o));
        PC2_TRY(encrypt_round(ctx, A->key, A->vq + o, nk, A->seed, A->round_ctr.p, 2, o, A->vhat, st, o));
        PC2_TRY(hom_add_at(ctx, A->key, A->zhat, A->vhat, nk, A->shat.p, st, o));
      }
      PC2_TRY(dispatch_to_mont(A, st));
      for (int k = 0; k < A->K; ++k)
        PC2_TRY(dispatch_matvec(A, A->tile_start[k], A->tile_start[k + 1] - A->tile_start[k], st));
      for (int k = 0; k < A->K; ++k) {
        const int o = A->off[k], nk = A->off[k + 1] - o;
        PC2_TRY(decrypt_at(ctx, A->key, A->xhat.p, nk, A->D.p, st, o));
      }
      PC2_TRY(launch_admm_update(A->D.p, A->Lh, A->N, A->node_of.p, A->node_size.p, A->brow.p, A->asum.p, A->mS,
                                 A->S, A->inv_s2, A->kappa, A->x.p, A->z.p, A->v.p, ctx->status, A->round_ctr.p,
                                 ctx->sms, st));
      continue;
    }
    if (!A->graph) {
      // first round eagerly (sizes the scratch), then capture one round for replay
      PC2_TRY(round_batched(A, st));
      if (cudaStreamSynchronize(st) != cudaSuccess) return PC2_ECUDA;
      if (!A->cap && cudaStreamCreateWithFlags(&A->cap, cudaStreamNonBlocking) != cudaSuccess) return PC2_ECUDA;
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(A->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return PC2_ECUDA;
      const int rc = round_batched(A, A->cap);
      const cudaError_t e = cudaStreamEndCapture(A->cap, &g);
      if (rc != PC2_OK) { if (g) cudaGraphDestroy(g); return rc; }
      if (e != cudaSuccess) return PC2_ECUDA;
      const cudaError_t ei = cudaGraphInstantiate(&A->graph, g, 0);
      cudaGraphDestroy(g);
      if (ei != cudaSuccess) { A->graph = nullptr; return PC2_ECUDA; }
      continue;
    }
    if (cudaGraphLaunch(A->graph, st) != cudaSuccess) return PC2_ECUDA;
  }
  return PC2_OK;
}

int pc2_admm_round_plain(pc2_admm* A, int rounds, pc2_stream_t stream) {
  if (!A || rounds < 0) return PC2_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  for (int r = 0; r < rounds; ++r) {
    PC2_TRY(launch_dis_xupdate(A->alpha.p, A->Bbar.p, A->boff.p, A->node_of.p, A->node_off.p, A->z.p, A->v.p, A->x.p,
                               A->N, A->ctx->sms, st));
    PC2_TRY(launch_zv_update(A->x.p, A->z.p, A->v.p, A->N, A->kappa, A->ctx->sms, st));
  }
  return PC2_OK;
}

int pc2_admm_get(pc2_admm* A, double* d_x, double* d_z, double* d_v, uint32_t* h_round, pc2_stream_t stream) {
  if (!A) return PC2_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  const size_t b = (size_t)A->N * 8;
  if ((d_x && cudaMemcpyAsync(d_x, A->x.p, b, cudaMemcpyDeviceToDevice, st)) ||
      (d_z && cudaMemcpyAsync(d_z, A->z.p, b, cudaMemcpyDeviceToDevice, st)) ||
      (d_v && cudaMemcpyAsync(d_v, A->v.p, b, cudaMemcpyDeviceToDevice, st)))
    return PC2_ECUDA;
  if (h_round) {
    if (cudaMemcpyAsync(h_round, A->round_ctr.p, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return PC2_ECUDA;
  }
  return PC2_OK;
}

int pc2_admm_set(pc2_admm* A, const double* d_x, const double* d_z, const double* d_v, uint32_t round,
                 pc2_stream_t stream) {
  if (!A || !d_x || !d_z || !d_v || round < 1) return PC2_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  const size_t b = (size_t)A->N * 8;
  if (cudaMemcpyAsync(A->x.p, d_x, b, cudaMemcpyDeviceToDevice, st) ||
      cudaMemcpyAsync(A->z.p, d_z, b, cudaMemcpyDeviceToDevice, st) ||
      cudaMemcpyAsync(A->v.p, d_v, b, cudaMemcpyDeviceToDevice, st) ||
      cudaMemcpyAsync(A->round_ctr.p, &round, 4, cudaMemcpyHostToDevice, st) || cudaStreamSynchronize(st))
    return PC2_ECUDA;
  return PC2_OK;
}

int pc2_admm_buffers(pc2_admm* A, const uint32_t** zhat, const uint32_t** vhat, const uint32_t** xhat,
                     const uint32_t** alpha_hat, const uint32_t** D, int* N) {
  if (!A) return PC2_EINVAL;
  if (zhat) *zhat = A->zhat;
  if (vhat) *vhat = A->vhat;
  if (xhat) *xhat = A->xhat.p;
  if (alpha_hat) *alpha_hat = A->alpha_hat.p;
  if (D) *D = A->D.p;
  if (N) *N = A->N;
  return PC2_OK;
}

int pc2_dequantize(pc2_ctx* ctx, const uint64_t* d_q, size_t n, double zmin, int log2_scale, int gamma, double* d_u,
                   pc2_stream_t stream) {
  if (!ctx || (n && (!d_q || !d_u)) || (gamma != 1 && gamma != 2) || log2_scale < 0 || log2_scale > 40)
    return PC2_EINVAL;
  if (!n) return PC2_OK;
  const double inv = std::ldexp(1.0, -(gamma == 1 ? 2 : 1) * log2_scale);
  return launch_dequantize(d_q, n, zmin, inv, d_u, ctx->sms, (cudaStream_t)stream);
}

int pc2_zv_update(pc2_ctx* ctx, const double* d_x, double* d_z, double* d_v, size_t n, double kappa,
                  pc2_stream_t stream) {
  if (!ctx || n > (size_t)0x7fffffff || (n && (!d_x || !d_z || !d_v)) || !(kappa >= 0.0)) return PC2_EINVAL;
  if (!n) return PC2_OK;
  return launch_zv_update(d_x, d_z, d_v, (int)n, kappa, ctx->sms, (cudaStream_t)stream);
}

int pc2_decode_matvec(pc2_ctx* ctx, const uint32_t* d_D, int limbs, size_t n, const long long* d_brow,
                      const unsigned long long* d_asum, const int* d_nk, double zmin, int log2_scale, double* d_x,
                      pc2_stream_t stream) {
  if (!ctx || limbs < 4 || limbs % 4 || log2_scale < 1 || log2_scale > 30 ||
      (n && (!d_D || !d_brow || !d_asum || !d_nk || !d_x)))
    return PC2_EINVAL;
  if (!n) return PC2_OK;
  const long long S = 1LL << log2_scale;
  const double ms = zmin * (double)S;
  if (ms != std::floor(ms) || std::fabs(ms) > 9.0e15) return PC2_EINVAL;  // zmin * S must be an integer
  return launch_decode_matvec(d_D, limbs, n, d_brow, d_asum, d_nk, (long long)ms, S, std::ldexp(1.0, -2 * log2_scale),
                              d_x, ctx->status, ctx->sms, (cudaStream_t)stream);
}

int pc2_hom_matvec(pc2_ctx* ctx, const pc2_key* key, const uint32_t* d_alpha, const uint32_t* d_s, const uint32_t* d_K,
                   size_t n, int kbits, uint32_t* d_out, pc2_stream_t stream) {
  if (!ctx || !key || kbits < 0 || kbits > 32 || n > (size_t)1 << 24 ||
      (n && (!d_alpha || !d_s || !d_K || !d_out)))
    return PC2_EINVAL;
  if (!n) return PC2_OK;
  const int kb = kbits ? kbits : 32;
  const cudaStream_t st = (cudaStream_t)stream;
  switch (2 * key->Lh) {
    case 16: return block_matvec_any<16>(ctx, key, d_alpha, d_s, d_K, (int)n, kb, d_out, st);
    case 32: return block_matvec_any<32>(ctx, key, d_alpha, d_s, d_K, (int)n, kb, d_out, st);
    case 64: return block_matvec_any<64>(ctx, key, d_alpha, d_s, d_K, (int)n, kb, d_out, st);
    case 128: return block_matvec_any<128>(ctx, key, d_alpha, d_s, d_K, (int)n, kb, d_out, st);
    case 192: return block_matvec_any<192>(ctx, key, d_alpha, d_s, d_K, (int)n, kb, d_out, st);
    case 256: return block_matvec_any<256>(ctx, key, d_alpha, d_s, d_K, (int)n, kb, d_out, st);
    default: return PC2_EUNSUPPORTED;
  }
}

int pc2_admm_save(pc2_admm* A, double* h_x, double* h_z, double* h_v, uint32_t* h_round) {
  if (!A || !h_x || !h_z || !h_v || !h_round) return PC2_EINVAL;
  const size_t b = (size_t)A->N * 8;
  if (cudaMemcpy(h_x, A->x.p, b, cudaMemcpyDeviceToHost) || cudaMemcpy(h_z, A->z.p, b, cudaMemcpyDeviceToHost) ||
      cudaMemcpy(h_v, A->v.p, b, cudaMemcpyDeviceToHost) ||
      cudaMemcpy(h_round, A->round_ctr.p, 4, cudaMemcpyDeviceToHost))
    return PC2_ECUDA;
  return PC2_OK;
}

int pc2_admm_load(pc2_admm* A, const double* h_x, const double* h_z, const double* h_v, uint32_t round) {
  if (!A || !h_x || !h_z || !h_v || round < 1) return PC2_EINVAL;
  const size_t b = (size_t)A->N * 8;
  if (cudaDeviceSynchronize() || cudaMemcpy(A->x.p, h_x, b, cudaMemcpyHostToDevice) ||
      cudaMemcpy(A->z.p, h_z, b, cudaMemcpyHostToDevice) || cudaMemcpy(A->v.p, h_v, b, cudaMemcpyHostToDevice) ||
      cudaMemcpy(A->round_ctr.p, &round, 4, cudaMemcpyHostToDevice))
    return PC2_ECUDA;
  return PC2_OK;
}

int pc2_admm_set_matvec(pc2_admm* A, int mode) {
  if (!A || mode < 0 || mode > 2) return PC2_EINVAL;
  if (A->graph) {
    cudaGraphExecDestroy(A->graph);
    A->graph = nullptr;
  }
  A->mv_mode = mode;
  return PC2_OK;
}

int pc2_admm_info(const pc2_admm* A, int* c, int* nwin, int* ntiles) {
  if (!A) return PC2_EINVAL;
  if (c) *c = A->c;
  if (nwin) *nwin = A->nwin;
  if (ntiles) *ntiles = A->ntiles;
  return PC2_OK;
}

}  // extern "C"
