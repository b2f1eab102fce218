// batch.cpp -- the batched form of the private ADMM round: many edge nodes,
// uneven node sizes, one key per key size, one persistent launch per round
// (k_batch_round) replayed as a CUDA graph, and the plain per-node path on
// the same state for comparison.
//
// Work items hold up to 128 / lanes consecutive elements of one node; they
// are ordered by their expected duration (longest first) so the persistent
// CTAs finish together.  Nodes of 2048-bit keys large enough for the
// tensor-core engine (PC2_TC_MIN_COUNT elements or more, engine automatic,
// or the engine forced to the tensor cores) hold no work items: a batched
// round runs them node by node through the per-operation entry points
// first, then the persistent launch over the other nodes, which advances
// the round counter for both.  The autotuner (pc2_batch_tune) times the window
// widths of each key's exponent schedules and the CTAs per SM on a sample
// of the work list without touching the state.
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
#include "pc2_batch.h"
#include "pc2_kernels.h"

namespace {

template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  int alloc(size_t count) {
    if (p) cudaFree(p);
    p = nullptr;
    n = count;
    if (!count) return PC2_OK;
    return cudaMalloc(&p, count * sizeof(T)) == cudaSuccess ? PC2_OK : PC2_ENOMEM;
  }
  ~DBuf() {
    if (p) cudaFree(p);
  }
};

#define PC2_TRYB(x)                  \
  do {                               \
    const int rc_ = (x);             \
    if (rc_ != PC2_OK) return rc_;   \
  } while (0)

}  // namespace

struct pc2_batch {
  pc2_ctx* ctx = nullptr;
  int K = 0;
  size_t N = 0;
  const pc2_key* key[pc2::kBatchClasses] = {};  // key per class
  int win_enc[pc2::kBatchClasses] = {};         // window widths in use (0 = automatic)
  int win_dec[pc2::kBatchClasses] = {};
  std::vector<pc2::BatchNode> nodes;
  std::vector<size_t> dct_off;                  // per node: word offset of its decrypted plaintexts (per-node path)
  std::vector<char> tc_node;                    // per node: runs on the tensor-core engine, not in the work list
  int tc_nodes = 0;
  double kappa = 0, zmin = 0, scale = 0, qmax = 0, inv_s2 = 0;
  long long mS = 0, S = 0;
  uint64_t seed = 0;
  size_t ct_words = 0, d_words = 0;
  DBuf<unsigned char> keyblk[pc2::kBatchClasses];
  DBuf<pc2::BatchConstMods> mods;
  DBuf<pc2::BatchNode> d_nodes;
  DBuf<pc2::BatchItem> d_items;
  DBuf<pc2::BatchCtl> ctl;
  DBuf<uint64_t> b, zq, vq;
  DBuf<uint32_t> alpha_hat, zhat, vhat, xhat, shat, that, D, scratch;
  DBuf<double> x, z, v;
  std::vector<pc2::BatchItem> items;
  int nitems = 0;
  int blocks_per_sm = 0;      // resident CTAs per SM (autotuned; <= occupancy limit)
  int grid = 0;
  size_t smem = 0, cta_words = 0;
  cudaGraphExec_t graph = nullptr;
  cudaStream_t cap = nullptr;
  ~pc2_batch() {
    if (graph) cudaGraphExecDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
  }
};

namespace pc2 {

// Expected duration of one work item of class c (relative): the element's
// products (proportional to Lh) times the product's cost per lane (Lh^2 / T).
static double item_cost(int cls) {
  const double Lh = kBatchLh[cls];
  return Lh * Lh * Lh / batch_lanes(kBatchLh[cls]);
}

template <int Lh>
static int build_key_block(pc2_batch* B, const pc2_key* key, int we, int wd, BatchConstMods* hm, int* tabw) {
  std::unique_ptr<BatchKey<Lh>> kb(new (std::nothrow) BatchKey<Lh>);
  if (!kb) return PC2_ENOMEM;
  std::memset(kb.get(), 0, sizeof(BatchKey<Lh>));
  PC2_TRYB(make_enc_crt<Lh>(*key, we, kb->enc));
  PC2_TRYB(make_dec<Lh>(*key, wd, kb->dec));
  fill_mod(kb->n2, key->n2);
  constexpr int c = batch_class(Lh);
  if constexpr (Lh <= 64) {
    uint32_t(*dst)[Lh] = nullptr;
    if constexpr (Lh == 8) dst = hm->m8;
    else if constexpr (Lh == 16) dst = hm->m16;
    else if constexpr (Lh == 32) dst = hm->m32;
    else dst = hm->m64;
    std::memcpy(dst[0], kb->enc.mp.n, sizeof(uint32_t) * Lh);
    std::memcpy(dst[1], kb->enc.mq.n, sizeof(uint32_t) * Lh);
    uint32_t(*hd)[Lh / 2] = nullptr;
    if constexpr (Lh == 8) hd = hm->h8;
    else if constexpr (Lh == 16) hd = hm->h16;
    else if constexpr (Lh == 32) hd = hm->h32;
    else hd = hm->h64;
    std::memcpy(hd[0], kb->enc.lp.h.n, sizeof(uint32_t) * (Lh / 2));
    std::memcpy(hd[1], kb->enc.lq.h.n, sizeof(uint32_t) * (Lh / 2));
  }
  const int w = std::max(std::max(kb->enc.ep.w, kb->enc.eq.w), std::max(kb->dec.ep.w, kb->dec.eq.w));
  *tabw = std::max((1 << (w - 1)) * Lh, (1 << 4) * 2 * Lh);  // CRT window tables; 16 entries mod n^2 (scaling)
  PC2_TRYB(B->keyblk[c].alloc(sizeof(BatchKey<Lh>)));
  if (cudaMemcpy(B->keyblk[c].p, kb.get(), sizeof(BatchKey<Lh>), cudaMemcpyHostToDevice) != cudaSuccess)
    return PC2_ECUDA;
  return PC2_OK;
}

// Key blocks, constant moduli, scratch and grid for the current windows and CTAs per SM.
static int batch_configure(pc2_batch* B, BatchParams* P) {
  BatchConstMods hm;
  std::memset(&hm, 0, sizeof(hm));
  std::memset(P, 0, sizeof(*P));
  size_t cta_words = 0, smem = 0;
  for (int c = 0; c < kBatchClasses; ++c) {
    if (!B->key[c]) continue;
    int tabw = 0;
    int rc = PC2_EUNSUPPORTED;
    switch (c) {
      case 0: rc = build_key_block<8>(B, B->key[c], B->win_enc[c], B->win_dec[c], &hm, &tabw); break;
      case 1: rc = build_key_block<16>(B, B->key[c], B->win_enc[c], B->win_dec[c], &hm, &tabw); break;
      case 2: rc = build_key_block<32>(B, B->key[c], B->win_enc[c], B->win_dec[c], &hm, &tabw); break;
      case 3: rc = build_key_block<64>(B, B->key[c], B->win_enc[c], B->win_dec[c], &hm, &tabw); break;
      case 4: rc = build_key_block<96>(B, B->key[c], B->win_enc[c], B->win_dec[c], &hm, &tabw); break;
    }
    if (rc != PC2_OK) return rc;
    const int Lh = kBatchLh[c], G = kThreads / batch_lanes(Lh);
    P->key[c] = B->keyblk[c].p;
    P->tabw[c] = tabw;
    cta_words = std::max(cta_words, (size_t)G * ((size_t)tabw + 10 * (size_t)(2 * Lh + 4)));
    smem = std::max(smem, (size_t)Lh * G * 4);
  }
  if (!B->mods.p) PC2_TRYB(B->mods.alloc(1));
  if (cudaMemcpy(B->mods.p, &hm, sizeof(hm), cudaMemcpyHostToDevice) != cudaSuccess) return PC2_ECUDA;
  const int per = batch_blocks_per_sm(smem);
  if (per < 1) return PC2_ECUDA;
  const int bps = B->blocks_per_sm > 0 ? std::min(B->blocks_per_sm, per) : per;
  const int grid = std::max(1, std::min(bps * B->ctx->sms, B->nitems));
  if (!B->scratch.p || B->scratch.n < (size_t)grid * cta_words) PC2_TRYB(B->scratch.alloc((size_t)grid * cta_words));
  B->grid = grid;
  B->smem = smem;
  B->cta_words = cta_words;
  P->nodes = B->d_nodes.p;
  P->items = B->d_items.p;
  P->nitems = (uint32_t)B->nitems;
  P->ctl = B->ctl.p;
  P->b = B->b.p;
  P->alpha_hat = B->alpha_hat.p;
  P->zhat = B->zhat.p;
  P->vhat = B->vhat.p;
  P->xhat = B->xhat.p;
  P->x = B->x.p;
  P->z = B->z.p;
  P->v = B->v.p;
  P->scratch = B->scratch.p;
  P->cta_words = cta_words;
  P->status = B->ctx->status;
  P->seed = B->seed;
  P->zmin = B->zmin;
  P->scale = B->scale;
  P->qmax = B->qmax;
  P->kappa = B->kappa;
  P->inv_s2 = B->inv_s2;
  P->mS = B->mS;
  P->S = B->S;
  return PC2_OK;
}

static void drop_graph(pc2_batch* B) {
  if (B->graph) cudaGraphExecDestroy(B->graph);
  B->graph = nullptr;
}

static int reset_state(pc2_batch* B, cudaStream_t st) {
  const BatchCtl c0{0u, 0u, 1u, 0u};
  if (cudaMemsetAsync(B->x.p, 0, B->N * 8, st) || cudaMemsetAsync(B->z.p, 0, B->N * 8, st) ||
      cudaMemsetAsync(B->v.p, 0, B->N * 8, st) ||
      cudaMemcpyAsync(B->ctl.p, &c0, sizeof(c0), cudaMemcpyHostToDevice, st) || cudaStreamSynchronize(st))
    return PC2_ECUDA;
  return PC2_OK;
}

// One round node by node through the per-operation entry points; with
// tc_only the tensor-core nodes alone, leaving the round counter to the
// persistent launch that follows.
static int per_node_round(pc2_batch* B, cudaStream_t st, bool tc_only = false) {
  pc2_ctx* ctx = B->ctx;
  if (!B->zq.p) {
    PC2_TRYB(B->zq.alloc(B->N));
    PC2_TRYB(B->vq.alloc(B->N));
    PC2_TRYB(B->shat.alloc(B->ct_words));
    PC2_TRYB(B->that.alloc(B->ct_words));
    PC2_TRYB(B->D.alloc(B->d_words));
  }
  uint32_t* round_ptr = reinterpret_cast<uint32_t*>(B->ctl.p) + 2;  // BatchCtl::round
  int last = B->K - 1;
  if (tc_only)
    while (last >= 0 && !B->tc_node[last]) --last;
  for (int k = 0; k <= last; ++k) {
    if (tc_only && !B->tc_node[k]) continue;
    const BatchNode& nd = B->nodes[k];
    const pc2_key* key = B->key[nd.cls];
    const size_t o = nd.elem0, n = nd.count;
    uint32_t* zh = B->zhat.p + nd.ct_off;
    uint32_t* vh = B->vhat.p + nd.ct_off;
    uint32_t* sh = B->shat.p + nd.ct_off;
    uint32_t* th = B->that.p + nd.ct_off;
    uint32_t* xh = B->xhat.p + nd.ct_off;
    uint32_t* Dk = B->D.p + B->dct_off[k];
    PC2_TRYB(launch_quantize(B->z.p + o, n, B->zmin, B->scale, B->qmax, 0, B->zq.p + o, ctx->status, nullptr,
                             ctx->sms, st));
    PC2_TRYB(launch_quantize(B->v.p + o, n, B->zmin, B->scale, B->qmax, 1, B->vq.p + o, ctx->status, nullptr,
                             ctx->sms, st));
    PC2_TRYB(encrypt_round(ctx, key, B->zq.p + o, n, B->seed, round_ptr, 1, o, zh, st));
    PC2_TRYB(encrypt_round(ctx, key, B->vq.p + o, n, B->seed, round_ptr, 2, o, vh, st));
    PC2_TRYB(hom_add_at(ctx, key, zh, vh, n, sh, st, 0));
    PC2_TRYB(pc2_hom_scal(ctx, key, sh, B->b.p + o, n, th, (pc2_stream_t)st));
    PC2_TRYB(hom_add_at(ctx, key, B->alpha_hat.p + nd.ct_off, th, n, xh, st, 0));
    PC2_TRYB(decrypt_at(ctx, key, xh, n, Dk, st, 0));
    PC2_TRYB(launch_batch_update(Dk, key->Lh, n, B->zq.p + o, B->vq.p + o, B->b.p + o, B->mS, B->S, B->inv_s2,
                                 B->kappa, B->x.p + o, B->z.p + o, B->v.p + o, ctx->status,
                                 !tc_only && k == last ? round_ptr : nullptr, ctx->sms, st));
  }
  return PC2_OK;
}

}  // namespace pc2

using namespace pc2;

extern "C" {

int pc2_batch_create(pc2_ctx* ctx, const pc2_batch_params* prm, const double* d_alpha, const double* d_bdiag,
                     pc2_batch** out, pc2_stream_t stream) {
  if (!ctx || !prm || !out || prm->nodes <= 0 || !prm->node_sizes || !prm->node_key || prm->nkeys <= 0 ||
      !prm->keys || !d_alpha || !d_bdiag)
    return PC2_EINVAL;
  *out = nullptr;
  if (!(prm->rho > 0) || !(prm->lambda >= 0) || !(prm->zmax > prm->zmin) || prm->log2_scale < 1 ||
      prm->log2_scale > 30)
    return PC2_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  std::unique_ptr<pc2_batch> B(new (std::nothrow) pc2_batch);
  if (!B) return PC2_ENOMEM;
  B->ctx = ctx;
  B->K = prm->nodes;
  // one key per key size
  std::vector<int> key_cls(prm->nkeys);
  for (int i = 0; i < prm->nkeys; ++i) {
    const pc2_key* k = prm->keys[i];
    if (!k) return PC2_EINVAL;
    if (!k->priv) return PC2_EKEY;
    const int c = batch_class(k->Lh);
    if (c < 0) return PC2_EUNSUPPORTED;
    if (B->key[c] && B->key[c] != k) return PC2_EINVAL;  // two different keys of one size
    B->key[c] = k;
    key_cls[i] = c;
  }
  B->kappa = prm->lambda / prm->rho;
  B->S = 1LL << prm->log2_scale;
  B->scale = (double)B->S;
  B->zmin = prm->zmin;
  const double ms = prm->zmin * B->scale;
  if (ms != std::floor(ms) || std::fabs(ms) > 9.0e15) return PC2_EINVAL;
  B->mS = (long long)ms;
  B->qmax = std::rint((prm->zmax - prm->zmin) * B->scale);
  B->inv_s2 = std::ldexp(1.0, -2 * prm->log2_scale);
  B->seed = prm->seed;
  // nodes, ciphertext offsets, work items
  size_t e0 = 0, ct = 0, dw = 0;
  for (int k = 0; k < B->K; ++k) {
    const int nk = prm->node_sizes[k], ki = prm->node_key[k];
    if (nk <= 0 || ki < 0 || ki >= prm->nkeys) return PC2_EINVAL;
    const int c = key_cls[ki], Lh = kBatchLh[c];
    BatchNode nd;
    nd.elem0 = e0;
    nd.ct_off = ct;
    nd.count = (uint32_t)nk;
    nd.cls = (uint32_t)c;
    B->nodes.push_back(nd);
    B->dct_off.push_back(dw);
    e0 += (size_t)nk;
    ct += pc2_tiled_words((size_t)nk, 2 * Lh);
    dw += pc2_tiled_words((size_t)nk, Lh);
    const bool tc = Lh == 64 && (ctx->engine == PC2_ENGINE_TC || (ctx->engine < 0 && nk >= PC2_TC_MIN_COUNT));
    B->tc_node.push_back(tc ? 1 : 0);
    B->tc_nodes += tc ? 1 : 0;
    const uint32_t G = (uint32_t)(kThreads / batch_lanes(Lh));
    for (uint32_t f = 0; !tc && f < (uint32_t)nk; f += G)
      B->items.push_back(BatchItem{(uint32_t)k, f, std::min(G, (uint32_t)nk - f), (uint32_t)c});
  }
  B->N = e0;
  B->ct_words = ct;
  B->d_words = dw;
  std::stable_sort(B->items.begin(), B->items.end(), [](const BatchItem& a, const BatchItem& b) {
    return item_cost((int)a.cls) > item_cost((int)b.cls);
  });
  B->nitems = (int)B->items.size();
  if (B->d_nodes.alloc(B->nodes.size()) || B->d_items.alloc(B->items.size()) || B->ctl.alloc(1) ||
      B->b.alloc(B->N) || B->x.alloc(B->N) || B->z.alloc(B->N) || B->v.alloc(B->N) ||
      B->alpha_hat.alloc(ct) || B->zhat.alloc(ct) || B->vhat.alloc(ct) || B->xhat.alloc(ct))
    return PC2_ENOMEM;
  if (cudaMemcpyAsync(B->d_nodes.p, B->nodes.data(), B->nodes.size() * sizeof(BatchNode), cudaMemcpyHostToDevice,
                      st) ||
      (!B->items.empty() && cudaMemcpyAsync(B->d_items.p, B->items.data(), B->items.size() * sizeof(BatchItem),
                                            cudaMemcpyHostToDevice, st)))
    return PC2_ECUDA;
  // b = Gamma2(Bbar_ii); alpha-hat = E(Gamma1(alpha)) per node with the node's key (r-stream 0)
  DBuf<uint64_t> c1;
  PC2_TRYB(c1.alloc(B->N));
  PC2_TRYB(launch_quantize(d_bdiag, B->N, B->zmin, B->scale, B->qmax, 0, B->b.p, ctx->status, nullptr, ctx->sms, st));
  PC2_TRYB(launch_quantize(d_alpha, B->N, B->zmin, B->scale * B->scale, B->qmax * B->scale, 0, c1.p, ctx->status,
                           nullptr, ctx->sms, st));
  for (int k = 0; k < B->K; ++k) {
    const BatchNode& nd = B->nodes[k];
    PC2_TRYB(pc2_encrypt(ctx, B->key[nd.cls], c1.p + nd.elem0, nd.count, B->seed, 0, nd.elem0,
                         B->alpha_hat.p + nd.ct_off, stream));
  }
  PC2_TRYB(reset_state(B.get(), st));
  BatchParams P;
  PC2_TRYB(batch_configure(B.get(), &P));
  *out = B.release();
  return PC2_OK;
}

void pc2_batch_destroy(pc2_batch* B) {
  if (!B) return;
  cudaSetDevice(B->ctx->device);
  cudaDeviceSynchronize();
  delete B;
}

int pc2_batch_reset(pc2_batch* B, pc2_stream_t stream) {
  if (!B) return PC2_EINVAL;
  return reset_state(B, (cudaStream_t)stream);
}

int pc2_batch_round(pc2_batch* B, int rounds, pc2_stream_t stream) {
  if (!B || rounds < 0) return PC2_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  if (!B->graph && rounds > 0) {
    BatchParams P;
    PC2_TRYB(batch_configure(B, &P));
    if (!B->cap && cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) != cudaSuccess) return PC2_ECUDA;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return PC2_ECUDA;
    const int rc = launch_batch_round(P, B->mods.p, B->smem, B->grid, B->cap);
    const cudaError_t e = cudaStreamEndCapture(B->cap, &g);
    if (rc != PC2_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return PC2_ECUDA;
    const cudaError_t ei = cudaGraphInstantiate(&B->graph, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      B->graph = nullptr;
      return PC2_ECUDA;
    }
  }
  for (int r = 0; r < rounds; ++r) {
    if (B->tc_nodes) PC2_TRYB(per_node_round(B, st, true));
    if (cudaGraphLaunch(B->graph, st) != cudaSuccess) return PC2_ECUDA;
  }
  return PC2_OK;
}

int pc2_batch_round_per_node(pc2_batch* B, int rounds, pc2_stream_t stream) {
  if (!B || rounds < 0) return PC2_EINVAL;
  for (int r = 0; r < rounds; ++r) PC2_TRYB(per_node_round(B, (cudaStream_t)stream));
  return PC2_OK;
}

int pc2_batch_get(pc2_batch* B, double* d_x, double* d_z, double* d_v, uint32_t* h_round, pc2_stream_t stream) {
  if (!B) return PC2_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  const size_t b = B->N * 8;
  if ((d_x && cudaMemcpyAsync(d_x, B->x.p, b, cudaMemcpyDeviceToDevice, st)) ||
      (d_z && cudaMemcpyAsync(d_z, B->z.p, b, cudaMemcpyDeviceToDevice, st)) ||
      (d_v && cudaMemcpyAsync(d_v, B->v.p, b, cudaMemcpyDeviceToDevice, st)))
    return PC2_ECUDA;
  if (h_round) {
    BatchCtl c;
    if (cudaMemcpyAsync(&c, B->ctl.p, sizeof(c), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return PC2_ECUDA;
    *h_round = c.round;
  }
  return PC2_OK;
}

int pc2_batch_ciphertexts(pc2_batch* B, int which, int node, const uint32_t** d_tiled, int* limbs) {
  if (!B || node < 0 || node >= B->K || !d_tiled || which < 0 || which > 3) return PC2_EINVAL;
  const BatchNode& nd = B->nodes[node];
  const uint32_t* pool = which == 0 ? B->alpha_hat.p : which == 1 ? B->zhat.p : which == 2 ? B->vhat.p : B->xhat.p;
  *d_tiled = pool + nd.ct_off;
  if (limbs) *limbs = 2 * kBatchLh[nd.cls];
  return PC2_OK;
}

int pc2_batch_info(const pc2_batch* B, size_t* elements, int* items, int* grid, size_t* scratch_bytes) {
  if (!B) return PC2_EINVAL;
  if (elements) *elements = B->N;
  if (items) *items = B->nitems;
  if (grid) *grid = B->grid;
  if (scratch_bytes) *scratch_bytes = B->scratch.n * 4;
  return PC2_OK;
}

int pc2_batch_tune(pc2_batch* B, int sample_items, pc2_stream_t stream, int* h_result) {
  if (!B || sample_items < 0) return PC2_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  if (cudaStreamSynchronize(st) != cudaSuccess) return PC2_ECUDA;
  // the sample: the first items of each class (in work-list order), at most sample_items in all
  const int per_sm_max = 3;
  std::vector<BatchItem> sample;
  {
    int counts[kBatchClasses] = {};
    int present = 0;
    for (int c = 0; c < kBatchClasses; ++c) present += B->key[c] ? 1 : 0;
    const int cap = sample_items > 0 ? sample_items : B->ctx->sms * per_sm_max;
    const int per_class = std::max(1, cap / std::max(1, present));
    for (const BatchItem& it : B->items)
      if (counts[it.cls] < per_class) {
        sample.push_back(it);
        ++counts[it.cls];
      }
  }
  if (sample.empty()) {  // every node on the tensor-core engine: nothing to tune
    if (h_result) {
      for (int c = 0; c < kBatchClasses; ++c) h_result[c] = B->key[c] ? B->win_enc[c] : 0;
      h_result[kBatchClasses] = B->blocks_per_sm;
    }
    return PC2_OK;
  }
  DBuf<BatchItem> d_sample;
  PC2_TRYB(d_sample.alloc(sample.size()));
  if (cudaMemcpy(d_sample.p, sample.data(), sample.size() * sizeof(BatchItem), cudaMemcpyHostToDevice) != cudaSuccess)
    return PC2_ECUDA;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto time_cfg = [&](float* ms) -> int {
    BatchParams P;
    PC2_TRYB(batch_configure(B, &P));
    P.items = d_sample.p;
    P.nitems = (uint32_t)sample.size();
    P.dry = 1;
    const int grid = std::max(1, std::min(B->grid, (int)sample.size()));
    cudaEventRecord(e0, st);
    PC2_TRYB(launch_batch_round(P, B->mods.p, B->smem, grid, st));
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) return PC2_ECUDA;
    cudaEventElapsedTime(ms, e0, e1);
    return PC2_OK;
  };
  int rc = PC2_OK;
  // window widths per present class (encryption and decryption together), then CTAs per SM
  for (int c = 0; c < kBatchClasses && rc == PC2_OK; ++c) {
    if (!B->key[c]) continue;
    float best = 1e30f;
    int bw = 0;
    for (int w = 4; w <= kMaxWin && rc == PC2_OK; ++w) {
      B->win_enc[c] = w;
      B->win_dec[c] = w;
      float ms = 0;
      rc = time_cfg(&ms);
      if (rc == PC2_OK && ms < best) {
        best = ms;
        bw = w;
      }
    }
    B->win_enc[c] = bw;
    B->win_dec[c] = bw;
  }
  float best = 1e30f;
  int bb = 0;
  for (int bps = 1; bps <= per_sm_max && rc == PC2_OK; ++bps) {
    B->blocks_per_sm = bps;
    float ms = 0;
    rc = time_cfg(&ms);
    // the sample is small: compare time per resident CTA slot filled
    if (rc == PC2_OK && ms < best) {
      best = ms;
      bb = bps;
    }
  }
  B->blocks_per_sm = bb;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != PC2_OK) return rc;
  drop_graph(B);
  BatchParams P;
  PC2_TRYB(batch_configure(B, &P));
  if (h_result) {
    for (int c = 0; c < kBatchClasses; ++c) h_result[c] = B->key[c] ? B->win_enc[c] : 0;
    h_result[kBatchClasses] = B->blocks_per_sm;
  }
  return PC2_OK;
}

}  // extern "C"
