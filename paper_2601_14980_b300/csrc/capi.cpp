// capi.cpp -- the extern "C" entry points of libpc2 (include/pc2.h).
//
// Marshals arguments, builds (and caches per key) the kernels' parameter
// blocks, owns the per-context scratch memory, and dispatches on the key size
// to the templated launchers.  No arithmetic on user data happens here.
#include <cuda_runtime.h>

#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <type_traits>
#include <utility>

#include "../../include/pc2.h"
#include "keys.hpp"
#include "philox.h"
#include "pc2_kernels.h"
#include "pc2_tc.h"

#include "ctx.hpp"

namespace pc2 {

// Parameter blocks cached per (key, kind, window): building them needs
// host big-integer work (inverses, schedules) that must stay off the hot path.
struct ParamCache {
  std::mutex mu;
  std::map<std::pair<const pc2_key*, int>, std::shared_ptr<void>> blocks;
};
static ParamCache& cache() {
  static ParamCache c;
  return c;
}
static void cache_drop(const pc2_key* k) {
  std::lock_guard<std::mutex> g(cache().mu);
  for (auto it = cache().blocks.begin(); it != cache().blocks.end();)
    it = it->first.first == k ? cache().blocks.erase(it) : std::next(it);
}

template <class P, class F>
static std::shared_ptr<P> cached(const pc2_key* k, int kind, int window, F make, int* rc) {
  const int tag = kind * 16 + window;
  {
    std::lock_guard<std::mutex> g(cache().mu);
    auto it = cache().blocks.find({k, tag});
    if (it != cache().blocks.end()) {
      *rc = PC2_OK;
      return std::static_pointer_cast<P>(it->second);
    }
  }
  std::shared_ptr<P> p(new (std::nothrow) P);
  if (!p) { *rc = PC2_ENOMEM; return nullptr; }
  *rc = make(*p);
  if (*rc != PC2_OK) return nullptr;
  std::lock_guard<std::mutex> g(cache().mu);
  cache().blocks[{k, tag}] = p;
  return p;
}

enum { KIND_ENC_CRT = 1, KIND_ENC_PUB = 2, KIND_DEC = 3, KIND_TC = 4, KIND_HOM = 64 };  // KIND_HOM + operands (1..32)

static uint32_t* ctx_scratch(void* c, size_t bytes) {
  pc2_ctx* ctx = static_cast<pc2_ctx*>(c);
  if (bytes <= ctx->scratch_bytes) return ctx->scratch;
  if (pc2_ctx_reserve(ctx, bytes) != PC2_OK) return nullptr;
  return ctx->scratch;
}

uint32_t* ctx_scratch_get(pc2_ctx* ctx, size_t bytes) { return ctx_scratch(ctx, bytes); }

// Lane counts built per operation and limb count (inst_crt_*.cu, inst_mv_*.cu).
const int* lane_set(int op, int limbs, int* n) {
  static const int s1[] = {1}, s124[] = {1, 2, 4}, s1248[] = {1, 2, 4, 8}, s248[] = {2, 4, 8}, s48[] = {4, 8};
  if (op == OP_MATVEC) {
    switch (limbs) {
      case 16: *n = 3; return s124;
      case 32: case 64: *n = 4; return s1248;
      case 128: case 192: case 256: *n = 2; return s48;
    }
  } else if (op == OP_N2) {  // first entry = lanes_for(limbs), the large-batch choice
    switch (limbs) {
      case 16: *n = 3; return s124;
      case 32: case 64: *n = 4; return s1248;
      case 128: case 192: case 256: *n = 2; return s48;
    }
  } else {
    switch (limbs) {
      case 8: *n = 3; return s124;
      case 16: case 32: case 64: *n = 4; return s1248;
      case 96: case 128: *n = 3; return s248;
    }
  }
  *n = 1;
  return s1;
}

static int log2_bucket(size_t count) {
  int b = 0;
  while (((size_t)1 << b) < count && b < 62) ++b;
  return b;
}

// Estimated time of one call with T lanes per element (halves split or not),
// in arbitrary units: the larger of
//   latency: waves x (halves run one after the other: 2, split: 1) x
//            (S + 64) per row -- a row's dependent chain grows with the
//            limbs per lane S = limbs / T, plus a fixed part (quotient
//            word, shuffles, loop) worth about 64 limbs;
//   issue:   count x 2 x limbs / SMs -- the instructions of all lanes, the
//            same for every T at this resolution.
// The constants were fitted to measured encryption + decryption times at
// 1024-, 2048- and 4096-bit n, 256..32768 elements, every lane count and
// both split modes; the chosen configuration was within 10 % of the fastest
// at every point.
static double lane_cost(int limbs, int T, bool split, size_t count, int sms) {
  const double cap = (double)sms * kThreads * min_blocks(limbs, T);
  const double waves = std::ceil((double)count * T * (split ? 2 : 1) / cap);
  const double lat = waves * (split ? 1.0 : 2.0) * ((double)limbs / T + 64.0) * 128.0;
  const double issue = (double)count * 2.0 * limbs / sms;
  return lat > issue ? lat : issue;
}

LaneCfg pick_config(pc2_ctx* ctx, int op, int limbs, size_t count) {
  int n = 0;
  const int* set = lane_set(op, limbs, &n);
  const bool can_split = op == OP_ENC_CRT || op == OP_DEC;
  const bool may_split = can_split && ctx->split != 1;
  const bool must_split = can_split && ctx->split == 2;
  {
    std::lock_guard<std::mutex> g(ctx->tune_mu);
    auto it = ctx->tuned.find(std::make_tuple(op, limbs, log2_bucket(count)));
    if (!ctx->lanes && it != ctx->tuned.end())
      return LaneCfg{std::get<0>(it->second), std::get<1>(it->second), std::get<2>(it->second) != 0};
  }
  if (op == OP_MATVEC) {
    // the most lanes per row that still fit one wave (about 384 threads per SM)
    const double cap = (double)ctx->sms * 384.0;
    if (ctx->lanes)
      for (int i = 0; i < n; ++i)
        if (set[i] == ctx->lanes) return LaneCfg{ctx->lanes, 0, false};
    LaneCfg best{set[0], 0, false};
    for (int i = 0; i < n; ++i)
      if ((double)count * set[i] <= cap) best = LaneCfg{set[i], 0, false};
    return best;
  }
  // forced lanes (when built for this size) fix T; otherwise every built T
  bool forced = false;
  for (int i = 0; i < n; ++i) forced = forced || set[i] == ctx->lanes;
  LaneCfg best{set[0], 0, must_split};
  double best_cost = 0.0;
  bool any = false;
  for (int i = 0; i < n; ++i) {
    if (forced && set[i] != ctx->lanes) continue;
    for (int s = 0; s < 2; ++s) {
      if ((s && !may_split) || (!s && must_split)) continue;
      const double c = lane_cost(limbs, set[i], s != 0, count, ctx->sms);
      if (!any || c < best_cost) {
        best = LaneCfg{set[i], 0, s != 0};
        best_cost = c;
        any = true;
      }
    }
  }
  return best;
}

template <int Lh, int T>
constexpr bool crt_has() {
  return (Lh == 8 && T <= 4) || ((Lh == 16 || Lh == 32 || Lh == 64) && T <= 8) ||
         ((Lh == 96 || Lh == 128) && T >= 2 && T <= 8);
}
// Calls fn(std::integral_constant<int, T>) for a built lane count T.
template <int Lh, class Fn>
static int with_crt_lanes(int T, Fn fn) {
  switch (T) {
    case 1: if constexpr (crt_has<Lh, 1>()) return fn(std::integral_constant<int, 1>()); break;
    case 2: if constexpr (crt_has<Lh, 2>()) return fn(std::integral_constant<int, 2>()); break;
    case 4: if constexpr (crt_has<Lh, 4>()) return fn(std::integral_constant<int, 4>()); break;
    case 8: if constexpr (crt_has<Lh, 8>()) return fn(std::integral_constant<int, 8>()); break;
  }
  return PC2_EUNSUPPORTED;
}

template <int L2, int T>
constexpr bool n2_has() {
  return (L2 == 16 && T <= 4) || ((L2 == 32 || L2 == 64) && T <= 8) ||
         ((L2 == 128 || L2 == 192 || L2 == 256) && (T == 4 || T == 8));
}
// Calls fn(std::integral_constant<int, T>) with the lane count picked for a
// power or product mod n^2 over `count` elements.
template <int L2, class Fn>
static int with_n2_lanes(pc2_ctx* ctx, size_t count, Fn fn) {
  switch (pick_config(ctx, OP_N2, L2, count).T) {
    case 1: if constexpr (n2_has<L2, 1>()) return fn(std::integral_constant<int, 1>()); break;
    case 2: if constexpr (n2_has<L2, 2>()) return fn(std::integral_constant<int, 2>()); break;
    case 4: if constexpr (n2_has<L2, 4>()) return fn(std::integral_constant<int, 4>()); break;
    case 8: if constexpr (n2_has<L2, 8>()) return fn(std::integral_constant<int, 8>()); break;
  }
  return PC2_EUNSUPPORTED;
}

// The tensor-core blocks of p^2 and q^2 (2048-bit keys), cached per key.
static std::shared_ptr<TcKeyMods> tc_mods(const pc2_key* key, int* rc) {
  return cached<TcKeyMods>(key, KIND_TC, 0, [&](TcKeyMods& K) {
    uint32_t w[64];
    mul(key->p, key->p).to_words(w, 64);
    if (!tc::build_mod<64>(w, K.p2)) return PC2_EKEY;
    mul(key->q, key->q).to_words(w, 64);
    if (!tc::build_mod<64>(w, K.q2)) return PC2_EKEY;
    key->p.to_words(w, 32);
    if (!tc::build_mod<32>(w, K.p)) return PC2_EKEY;
    key->q.to_words(w, 32);
    if (!tc::build_mod<32>(w, K.q)) return PC2_EKEY;
    return PC2_OK;
  }, rc);
}
static bool use_tc(const pc2_ctx* ctx, size_t count) {
  return ctx->engine == PC2_ENGINE_TC || (ctx->engine < 0 && count >= (size_t)PC2_TC_MIN_COUNT);
}

template <int Lh>
static int enc_crt(pc2_ctx* ctx, const pc2_key* key, const uint64_t* m64, const uint32_t* mw, size_t count,
                   uint64_t seed, uint32_t stream, uint64_t e0, uint32_t* out, cudaStream_t st) {
  const LaneCfg cfg = pick_config(ctx, OP_ENC_CRT, Lh, count);
  const int w = cfg.w ? cfg.w : ctx->window;
  int rc;
  auto P0 = cached<EncCrtParams<Lh>>(key, KIND_ENC_CRT, w,
                                     [&](EncCrtParams<Lh>& P) { return make_enc_crt<Lh>(*key, w, P); }, &rc);
  if (!P0) return rc;
  std::unique_ptr<EncCrtParams<Lh>> P(new (std::nothrow) EncCrtParams<Lh>(*P0));
  if (!P) return PC2_ENOMEM;
  P->seed = seed;
  P->stream = stream;
  P->e0 = e0;
  P->mwords = mw ? Lh : 2;
  if constexpr (Lh == 64) {
    if (use_tc(ctx, count)) {
      auto K = tc_mods(key, &rc);
      if (!K) return rc;
      ctx->ev_recorded = ctx->timing;
      return launch_enc_crt_tc(*P, *K, m64, mw, count, out, ctx_scratch, ctx, ctx->status, ctx->sms, st, 0,
                               ctx->timing ? ctx->ev : nullptr);
    }
  }
  return with_crt_lanes<Lh>(cfg.T, [&](auto tt) {
    constexpr int T = decltype(tt)::value;
    if (cfg.split) return launch_enc_crt2<Lh, T>(*P, m64, mw, count, out, ctx_scratch, ctx, ctx->status, ctx->sms, st, 0);
    return launch_enc_crt<Lh, T>(*P, m64, mw, count, out, ctx_scratch, ctx, ctx->status, ctx->sms, st, 0);
  });
}

template <int Lh>
static int enc_crt_round(pc2_ctx* ctx, const pc2_key* key, const uint64_t* m64, size_t count, uint64_t seed,
                         const uint32_t* round_ptr, uint32_t kind, uint64_t e0, uint32_t* out, cudaStream_t st,
                         size_t base, size_t split, uint32_t kind2, size_t base2) {
  const LaneCfg cfg = pick_config(ctx, OP_ENC_CRT, Lh, count);
  const int w = cfg.w ? cfg.w : ctx->window;
  int rc;
  auto P0 = cached<EncCrtParams<Lh>>(key, KIND_ENC_CRT, w,
                                     [&](EncCrtParams<Lh>& P) { return make_enc_crt<Lh>(*key, w, P); }, &rc);
  if (!P0) return rc;
  std::unique_ptr<EncCrtParams<Lh>> P(new (std::nothrow) EncCrtParams<Lh>(*P0));
  if (!P) return PC2_ENOMEM;
  P->seed = seed;
  P->e0 = e0;
  P->mwords = 2;
  P->round_ptr = round_ptr;
  P->kind = kind;
  P->split = split;
  P->kind2 = kind2;
  P->base2 = base2;
  if constexpr (Lh == 64) {
    // the tensor-core engine per vector (elements [0, split) with stream
    // kind, the rest with kind2 at counter e0 + (e - split), output base2)
    const size_t n1 = split < count ? split : count, n2 = count - n1;
    if (use_tc(ctx, n1 > n2 ? n1 : n2)) {
      auto K = tc_mods(key, &rc);
      if (!K) return rc;
      rc = n1 ? launch_enc_crt_tc(*P, *K, m64, nullptr, n1, out, ctx_scratch, ctx, ctx->status, ctx->sms, st, base,
                                  nullptr)
              : PC2_OK;
      if (rc != PC2_OK || !n2) return rc;
      P->kind = kind2;
      return launch_enc_crt_tc(*P, *K, m64 + n1, nullptr, n2, out, ctx_scratch, ctx, ctx->status, ctx->sms, st,
                               base2, nullptr);
    }
  }
  return with_crt_lanes<Lh>(cfg.T, [&](auto tt) {
    constexpr int T = decltype(tt)::value;
    if (cfg.split)  // both vectors in one launch
      return launch_enc_crt2<Lh, T>(*P, m64, nullptr, count, out, ctx_scratch, ctx, ctx->status, ctx->sms, st, base);
    if (split >= count)
      return launch_enc_crt<Lh, T>(*P, m64, nullptr, count, out, ctx_scratch, ctx, ctx->status, ctx->sms, st, base);
    // the one-vector kernel: the two vectors one after the other
    int r = launch_enc_crt<Lh, T>(*P, m64, nullptr, split, out, ctx_scratch, ctx, ctx->status, ctx->sms, st, base);
    if (r != PC2_OK) return r;
    P->kind = kind2;
    return launch_enc_crt<Lh, T>(*P, m64 + split, nullptr, count - split, out, ctx_scratch, ctx, ctx->status,
                                 ctx->sms, st, base2);
  });
}

int encrypt_round(pc2_ctx* ctx, const pc2_key* key, const uint64_t* d_m, size_t count, uint64_t seed,
                  const uint32_t* round_ptr, uint32_t kind, uint64_t e0, uint32_t* d_ct, cudaStream_t st,
                  size_t base, size_t split, uint32_t kind2, size_t base2) {
  if (!ctx || !key || !key->priv) return PC2_EKEY;
  if (!count) return PC2_OK;
#define PC2_CALL_ROUND(L) \
  enc_crt_round<L>(ctx, key, d_m, count, seed, round_ptr, kind, e0, d_ct, st, base, split, kind2, base2)
  switch (key->Lh) {
    case 8: return PC2_CALL_ROUND(8);
    case 16: return PC2_CALL_ROUND(16);
    case 32: return PC2_CALL_ROUND(32);
    case 64: return PC2_CALL_ROUND(64);
    case 96: return PC2_CALL_ROUND(96);
    case 128: return PC2_CALL_ROUND(128);
    default: return PC2_EUNSUPPORTED;
  }
#undef PC2_CALL_ROUND
}

template <int L2>
static int enc_pub(pc2_ctx* ctx, const pc2_key* key, const uint64_t* m64, const uint32_t* mw, size_t count,
                   uint64_t seed, uint32_t stream, uint64_t e0, uint32_t* out, cudaStream_t st) {
  int rc;
  auto P0 = cached<EncPubParams<L2>>(key, KIND_ENC_PUB, ctx->window,
                                     [&](EncPubParams<L2>& P) { return make_enc_pub<L2>(*key, ctx->window, P); }, &rc);
  if (!P0) return rc;
  std::unique_ptr<EncPubParams<L2>> P(new (std::nothrow) EncPubParams<L2>(*P0));
  if (!P) return PC2_ENOMEM;
  P->seed = seed;
  P->stream = stream;
  P->e0 = e0;
  P->mwords = mw ? L2 / 2 : 2;
  return with_n2_lanes<L2>(ctx, count, [&](auto tt) {
    return launch_enc_pub<L2, decltype(tt)::value>(*P, m64, mw, count, out, ctx_scratch, ctx, ctx->status, ctx->sms, st);
  });
}

template <int Lh>
static int dec(pc2_ctx* ctx, const pc2_key* key, const uint32_t* ct, size_t count, uint32_t* out, cudaStream_t st,
               size_t base = 0) {
  const LaneCfg cfg = pick_config(ctx, OP_DEC, Lh, count);
  const int w = cfg.w ? cfg.w : ctx->window;
  int rc;
  auto P = cached<DecParams<Lh>>(key, KIND_DEC, w, [&](DecParams<Lh>& p) { return make_dec<Lh>(*key, w, p); }, &rc);
  if (!P) return rc;
  if constexpr (Lh == 64) {
    if (use_tc(ctx, count)) {
      auto K = tc_mods(key, &rc);
      if (!K) return rc;
      ctx->ev_recorded = ctx->timing;
      return launch_dec_crt_tc(*P, *K, ct, count, out, ctx_scratch, ctx, ctx->status, ctx->sms, st, base,
                               ctx->timing ? ctx->ev : nullptr);
    }
  }
  return with_crt_lanes<Lh>(cfg.T, [&](auto tt) {
    constexpr int T = decltype(tt)::value;
    if (cfg.split) return launch_dec_crt2<Lh, T>(*P, ct, count, out, ctx_scratch, ctx, ctx->sms, st, base);
    return launch_dec_crt<Lh, T>(*P, ct, count, out, ctx_scratch, ctx, ctx->sms, st, base);
  });
}

template <int Lh>
std::shared_ptr<DecParams<Lh>> dec_params(const pc2_key* key, int* rc) {
  return cached<DecParams<Lh>>(key, KIND_DEC, 0, [&](DecParams<Lh>& p) { return make_dec<Lh>(*key, 0, p); }, rc);
}
template std::shared_ptr<DecParams<8>> dec_params<8>(const pc2_key*, int*);
template std::shared_ptr<DecParams<16>> dec_params<16>(const pc2_key*, int*);
template std::shared_ptr<DecParams<32>> dec_params<32>(const pc2_key*, int*);
template std::shared_ptr<DecParams<64>> dec_params<64>(const pc2_key*, int*);
template std::shared_ptr<DecParams<96>> dec_params<96>(const pc2_key*, int*);
template std::shared_ptr<DecParams<128>> dec_params<128>(const pc2_key*, int*);

template <int Lh>
std::shared_ptr<EncCrtParams<Lh>> enc_params(const pc2_key* key, int* rc) {
  return cached<EncCrtParams<Lh>>(key, KIND_ENC_CRT, 0,
                                  [&](EncCrtParams<Lh>& p) { return make_enc_crt<Lh>(*key, 0, p); }, rc);
}
template std::shared_ptr<EncCrtParams<8>> enc_params<8>(const pc2_key*, int*);
template std::shared_ptr<EncCrtParams<16>> enc_params<16>(const pc2_key*, int*);
template std::shared_ptr<EncCrtParams<32>> enc_params<32>(const pc2_key*, int*);
template std::shared_ptr<EncCrtParams<64>> enc_params<64>(const pc2_key*, int*);

template <int L2>
static int hom_sum(pc2_ctx* ctx, const pc2_key* key, const uint32_t* const* srcs, size_t groups, size_t count,
                   uint32_t* out, cudaStream_t st, size_t base = 0) {
  // chunks of at most kMaxGroups operands; later chunks start from the running product
  size_t done = 0;
  bool first = true;
  while (done < groups) {
    int k = 0;
    const uint32_t* ops[kMaxGroups];
    if (!first) ops[k++] = out;
    while (k < kMaxGroups && done < groups) ops[k++] = srcs[done++];
    int rc;
    auto P0 = cached<HomParams<L2>>(key, KIND_HOM + k, 0, [&](HomParams<L2>& p) { return make_hom<L2>(*key, 0, k, p); },
                                    &rc);
    if (!P0) return rc;
    std::unique_ptr<HomParams<L2>> P(new (std::nothrow) HomParams<L2>(*P0));
    if (!P) return PC2_ENOMEM;
    for (int i = 0; i < k; ++i) P->src[i] = ops[i];
    rc = with_n2_lanes<L2>(ctx, count, [&](auto tt) {
      return launch_hom_sum<L2, decltype(tt)::value>(*P, count, out, ctx->sms, st, base);
    });
    if (rc) return rc;
    first = false;
  }
  return PC2_OK;
}

int hom_add_at(pc2_ctx* ctx, const pc2_key* key, const uint32_t* a, const uint32_t* b, size_t count, uint32_t* out,
               cudaStream_t st, size_t base) {
  if (!count) return PC2_OK;
  const uint32_t* srcs[2] = {a, b};
  switch (key->Lh) {
    case 8: return hom_sum<16>(ctx, key, srcs, 2, count, out, st, base);
    case 16: return hom_sum<32>(ctx, key, srcs, 2, count, out, st, base);
    case 32: return hom_sum<64>(ctx, key, srcs, 2, count, out, st, base);
    case 64: return hom_sum<128>(ctx, key, srcs, 2, count, out, st, base);
    case 96: return hom_sum<192>(ctx, key, srcs, 2, count, out, st, base);
    case 128: return hom_sum<256>(ctx, key, srcs, 2, count, out, st, base);
    default: return PC2_EUNSUPPORTED;
  }
}

int decrypt_at(pc2_ctx* ctx, const pc2_key* key, const uint32_t* ct, size_t count, uint32_t* out, cudaStream_t st,
               size_t base) {
  if (!key->priv) return PC2_EKEY;
  if (!count) return PC2_OK;
  switch (key->Lh) {
    case 8: return dec<8>(ctx, key, ct, count, out, st, base);
    case 16: return dec<16>(ctx, key, ct, count, out, st, base);
    case 32: return dec<32>(ctx, key, ct, count, out, st, base);
    case 64: return dec<64>(ctx, key, ct, count, out, st, base);
    case 96: return dec<96>(ctx, key, ct, count, out, st, base);
    case 128: return dec<128>(ctx, key, ct, count, out, st, base);
    default: return PC2_EUNSUPPORTED;
  }
}

template <int L2>
static int hom_scal(pc2_ctx* ctx, const pc2_key* key, const uint32_t* ct, const uint64_t* k, size_t count,
                    uint32_t* out, cudaStream_t st) {
  const int w = ctx->window ? (ctx->window > 5 ? 5 : ctx->window) : 4;
  int rc;
  auto P = cached<HomParams<L2>>(key, KIND_HOM + 1, w, [&](HomParams<L2>& p) { return make_hom<L2>(*key, w, 1, p); },
                                 &rc);
  if (!P) return rc;
  return with_n2_lanes<L2>(ctx, count, [&](auto tt) {
    return launch_hom_scal<L2, decltype(tt)::value>(*P, ct, k, count, out, ctx_scratch, ctx, ctx->sms, st);
  });
}

// Window of a full-width scalar: the context's width clamped to 4..6, else 5.
template <int L2>
static int hom_scal_wide(pc2_ctx* ctx, const pc2_key* key, const uint32_t* ct, const uint32_t* kw, size_t count,
                         uint32_t* out, cudaStream_t st) {
  const int w = ctx->window ? (ctx->window < 4 ? 4 : (ctx->window > 6 ? 6 : ctx->window)) : 5;
  int rc;
  auto P = cached<HomParams<L2>>(key, KIND_HOM + 1, w, [&](HomParams<L2>& p) { return make_hom<L2>(*key, w, 1, p); },
                                 &rc);
  if (!P) return rc;
  return with_n2_lanes<L2>(ctx, count, [&](auto tt) {
    return launch_hom_scal_wide<L2, decltype(tt)::value>(*P, ct, kw, count, out, ctx_scratch, ctx, ctx->sms, st);
  });
}

}  // namespace pc2

using namespace pc2;

#define PC2_DISPATCH_H(Lh, call) \
  switch (Lh) {                  \
    case 8: return call(8);      \
    case 16: return call(16);    \
    case 32: return call(32);    \
    case 64: return call(64);    \
    case 96: return call(96);    \
    case 128: return call(128);  \
    default: return PC2_EUNSUPPORTED; \
  }

extern "C" {

const char* pc2_strerror(int code) {
  switch (code) {
    case PC2_OK: return "ok";
    case PC2_EINVAL: return "invalid argument";
    case PC2_ERANGE: return "value out of range";
    case PC2_EKEY: return "invalid key or private-key operation on a public key";
    case PC2_ENOMEM: return "out of memory";
    case PC2_ECUDA: return "CUDA error";
    case PC2_ETIMEOUT: return "timed out";
    case PC2_EMISSING: return "missing input";
    case PC2_EUNSUPPORTED: return "unsupported configuration";
    default: return "unknown error";
  }
}

int pc2_ctx_create(int device, pc2_ctx** out) {
  if (!out) return PC2_EINVAL;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return PC2_ECUDA;
  std::unique_ptr<pc2_ctx> c(new (std::nothrow) pc2_ctx);
  if (!c) return PC2_ENOMEM;
  c->device = device;
  if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return PC2_ECUDA;
  if (cudaMalloc(&c->status, sizeof(int)) != cudaSuccess) return PC2_ENOMEM;
  if (cudaMemset(c->status, 0, sizeof(int)) != cudaSuccess) return PC2_ECUDA;
  *out = c.release();
  return PC2_OK;
}

void pc2_ctx_destroy(pc2_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->scratch) cudaFree(ctx->scratch);
  if (ctx->status) cudaFree(ctx->status);
  for (auto& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  delete ctx;
}

int pc2_ctx_reserve(pc2_ctx* ctx, size_t bytes) {
  if (!ctx) return PC2_EINVAL;
  if (bytes <= ctx->scratch_bytes) return PC2_OK;
  const size_t gran = (size_t)64 << 20;
  bytes = (bytes + gran - 1) / gran * gran;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return PC2_ECUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return PC2_ECUDA;  // earlier users of the old buffer
  if (ctx->scratch) cudaFree(ctx->scratch);
  ctx->scratch = nullptr;
  ctx->scratch_bytes = 0;
  if (cudaMalloc(&ctx->scratch, bytes) != cudaSuccess) {
    ctx->scratch = nullptr;
    return PC2_ENOMEM;
  }
  ctx->scratch_bytes = bytes;
  return PC2_OK;
}

size_t pc2_ctx_scratch_bytes(const pc2_ctx* ctx) { return ctx ? ctx->scratch_bytes : 0; }

int pc2_ctx_status(pc2_ctx* ctx, pc2_stream_t stream, int* bits) {
  if (!ctx || !bits) return PC2_EINVAL;
  int v = 0;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return PC2_ECUDA;
  if (cudaMemcpy(&v, ctx->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return PC2_ECUDA;
  if (cudaMemset(ctx->status, 0, sizeof(int)) != cudaSuccess) return PC2_ECUDA;
  *bits = v;
  return PC2_OK;
}

int pc2_ctx_set_window(pc2_ctx* ctx, int w) {
  if (!ctx || (w != 0 && (w < 3 || w > kMaxWin))) return PC2_EINVAL;
  ctx->window = w;
  return PC2_OK;
}

int pc2_ctx_set_lanes(pc2_ctx* ctx, int lanes) {
  if (!ctx || (lanes != 0 && lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8)) return PC2_EINVAL;
  ctx->lanes = lanes;
  return PC2_OK;
}

int pc2_ctx_set_split(pc2_ctx* ctx, int mode) {
  if (!ctx || mode < 0 || mode > 2) return PC2_EINVAL;
  ctx->split = mode;
  return PC2_OK;
}

int pc2_ctx_set_engine(pc2_ctx* ctx, int engine) {
  if (!ctx || (engine != -1 && engine != PC2_ENGINE_IMAD && engine != PC2_ENGINE_TC)) return PC2_EINVAL;
  ctx->engine = engine;
  return PC2_OK;
}

int pc2_ctx_set_timing(pc2_ctx* ctx, int on) {
  if (!ctx) return PC2_EINVAL;
  if (on && !ctx->ev[0])
    for (auto& e : ctx->ev)
      if (cudaEventCreate(&e) != cudaSuccess) return PC2_ECUDA;
  ctx->timing = on != 0;
  ctx->ev_recorded = false;
  return PC2_OK;
}

int pc2_ctx_stage_ms(pc2_ctx* ctx, double* h_ms) {
  if (!ctx || !h_ms) return PC2_EINVAL;
  if (!ctx->ev_recorded) return PC2_EINVAL;
  if (cudaEventSynchronize(ctx->ev[4]) != cudaSuccess) return PC2_ECUDA;
  for (int i = 0; i < 4; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->ev[i], ctx->ev[i + 1]) != cudaSuccess) return PC2_ECUDA;
    h_ms[i] = ms;
  }
  return PC2_OK;
}

int pc2_key_power_counts(const pc2_key* key, int op, long* squarings, long* multiplies, int* limbs) {
  if (!key || !squarings || !multiplies || !limbs || (op != 0 && op != 2)) return PC2_EINVAL;
  if (!key->priv) return PC2_EKEY;
  auto count = [&](const auto& E, long& sq, long& mu) {
    const int ntab = 1 << (E.w - 1);
    if (ntab > 1) {
      sq += 1;
      mu += ntab - 1;
    }
    for (int i = 1; i < E.nsteps; ++i) {
      sq += E.step[i] >> 8;
      mu += ((E.step[i] & 0xffu) != 0u) ? 1 : 0;
    }
  };
  *squarings = 0;
  *multiplies = 0;
  int rc = PC2_OK;
  auto fill = [&](auto tag) -> int {
    constexpr int Lh = decltype(tag)::value;
    if (op == 0) {
      auto P = enc_params<Lh>(key, &rc);
      if (!P) return rc;
      if constexpr (lift_route<Lh, 1>()) {
        count(P->lp.e2, *squarings, *multiplies);
        count(P->lq.e2, *squarings, *multiplies);
      } else {
        count(P->ep, *squarings, *multiplies);
        count(P->eq, *squarings, *multiplies);
      }
    } else {
      auto P = dec_params<Lh>(key, &rc);
      if (!P) return rc;
      count(P->ep, *squarings, *multiplies);
      count(P->eq, *squarings, *multiplies);
    }
    *limbs = Lh;
    return PC2_OK;
  };
  switch (key->Lh) {
    case 8: return fill(std::integral_constant<int, 8>());
    case 16: return fill(std::integral_constant<int, 16>());
    case 32: return fill(std::integral_constant<int, 32>());
    case 64: return fill(std::integral_constant<int, 64>());
    default: return PC2_EUNSUPPORTED;
  }
}

int pc2_autotune(pc2_ctx* ctx, const pc2_key* key, size_t count, int ops, pc2_stream_t stream, int* h_result) {
  if (!ctx || !key || !count || (ops & ~3) || !ops) return PC2_EINVAL;
  if (!key->priv) return PC2_EKEY;
  const cudaStream_t st = (cudaStream_t)stream;
  const int Lh = key->Lh;
  // time at most two resident waves; larger counts of the same size class
  // behave the same per wave
  const size_t cap = (size_t)ctx->sms * 384 * 2;
  const size_t n = count < cap ? count : cap;
  uint64_t* dm = nullptr;
  uint32_t *dct = nullptr, *dout = nullptr;
  if (cudaMalloc(&dm, n * 8) != cudaSuccess) return PC2_ENOMEM;
  if (cudaMalloc(&dct, pc2_tiled_words(n, 2 * Lh) * 4) != cudaSuccess ||
      cudaMalloc(&dout, pc2_tiled_words(n, Lh) * 4) != cudaSuccess) {
    cudaFree(dm);
    cudaFree(dct);
    return PC2_ENOMEM;
  }
  cudaMemsetAsync(dm, 0x5a, n * 8, st);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int saved_lanes = ctx->lanes, saved_window = ctx->window, saved_split = ctx->split;
  int rc = PC2_OK, res_i = 0;
  for (int op : {OP_ENC_CRT, OP_DEC}) {
    if (!((op == OP_ENC_CRT && (ops & 1)) || (op == OP_DEC && (ops & 2)))) continue;
    int nl = 0;
    const int* set = lane_set(op, Lh, &nl);
    // decryption times the ciphertexts of an encryption pass
    if (op == OP_DEC) {
      ctx->lanes = 0;
      ctx->window = saved_window;
      ctx->split = saved_split;
      rc = pc2_encrypt(ctx, key, dm, n, 1, 1, 0, dct, stream);
      if (rc != PC2_OK) break;
    }
    float best = 1e30f;
    std::tuple<int, int, int> pick{set[0], 0, 0};
    for (int i = 0; i < nl && rc == PC2_OK; ++i) {
      for (int s = 0; s < 2 && rc == PC2_OK; ++s) {
        for (int w = 4; w <= kMaxWin && rc == PC2_OK; ++w) {
          ctx->lanes = set[i];
          ctx->split = s ? 2 : 1;
          ctx->window = w;
          cudaEventRecord(e0, st);
          rc = op == OP_ENC_CRT ? pc2_encrypt(ctx, key, dm, n, 1, 1, 0, dct, stream)
                                : pc2_decrypt(ctx, key, dct, n, dout, stream);
          cudaEventRecord(e1, st);
          if (cudaEventSynchronize(e1) != cudaSuccess) rc = PC2_ECUDA;
          float ms = 0;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rc == PC2_OK && ms < best) {
            best = ms;
            pick = std::make_tuple(set[i], w, s);
          }
        }
      }
    }
    if (rc != PC2_OK) break;
    {
      std::lock_guard<std::mutex> g(ctx->tune_mu);
      ctx->tuned[std::make_tuple(op, Lh, log2_bucket(count))] = pick;
    }
    if (h_result) {
      h_result[res_i++] = std::get<0>(pick);
      h_result[res_i++] = std::get<1>(pick);
      h_result[res_i++] = std::get<2>(pick);
    }
  }
  ctx->lanes = saved_lanes;
  ctx->window = saved_window;
  ctx->split = saved_split;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  cudaFree(dm);
  cudaFree(dct);
  cudaFree(dout);
  return rc;
}

int pc2_keygen(int nbits, uint64_t seed, pc2_key** out) {
  if (!out || !supported_nbits(nbits)) return PC2_EINVAL;
  *out = nullptr;
  const int half = nbits / 2;
  Big pr[2];
  uint32_t cand = 0;
  for (int which = 0; which < 2;) {
    Big x;
    x.w.assign((size_t)half / 32, 0);
    for (size_t j = 0; j < x.w.size(); j += 4) {
      const U4 v = philox4x32_10(U4{(uint32_t)j, cand, (uint32_t)nbits, 0x6B657967u}, (uint32_t)seed,
                                 (uint32_t)(seed >> 32));
      const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
      for (int i = 0; i < 4 && j + i < x.w.size(); ++i) x.w[j + i] = w4[i];
    }
    ++cand;
    x.w.back() |= 0xC0000000u;  // top two bits: p q has exactly nbits bits
    x.w[0] |= 1u;
    if (!probable_prime(x, 32, seed ^ cand)) continue;
    if (which == 1 && cmp(x, pr[0]) == 0) continue;
    pr[which++] = x;
  }
  return key_from_primes(pr[0], pr[1], out);
}

int pc2_key_from_primes(const uint32_t* h_p, const uint32_t* h_q, int words, pc2_key** out) {
  if (!h_p || !h_q || words <= 0 || !out) return PC2_EINVAL;
  *out = nullptr;
  try {
    return key_from_primes(Big::from_words(h_p, (size_t)words), Big::from_words(h_q, (size_t)words), out);
  } catch (...) {
    return PC2_EINVAL;
  }
}

int pc2_key_public(const pc2_key* key, pc2_key** out) {
  if (!key || !out) return PC2_EINVAL;
  std::unique_ptr<pc2_key> k(new (std::nothrow) pc2_key);
  if (!k) return PC2_ENOMEM;
  k->nbits = key->nbits;
  k->Lh = key->Lh;
  k->priv = false;
  k->n = key->n;
  k->n2 = key->n2;
  *out = k.release();
  return PC2_OK;
}

void pc2_key_destroy(pc2_key* key) {
  if (!key) return;
  cache_drop(key);
  delete key;
}

int pc2_key_info(const pc2_key* key, int* nbits, int* has_private) {
  if (!key) return PC2_EINVAL;
  if (nbits) *nbits = key->nbits;
  if (has_private) *has_private = key->priv ? 1 : 0;
  return PC2_OK;
}

int pc2_key_export(const pc2_key* key, uint32_t* h_n, uint32_t* h_p, uint32_t* h_q, uint32_t* h_lambda, uint32_t* h_mu) {
  if (!key) return PC2_EINVAL;
  if (h_n) key->n.to_words(h_n, key->Lh);
  if ((h_p || h_q || h_lambda || h_mu) && !key->priv) return PC2_EKEY;
  if (h_p) key->p.to_words(h_p, key->Lh / 2);
  if (h_q) key->q.to_words(h_q, key->Lh / 2);
  if (h_lambda) key->lambda.to_words(h_lambda, key->Lh);
  if (h_mu) key->mu.to_words(h_mu, key->Lh);
  return PC2_OK;
}

int pc2_key_cost(const pc2_ctx* ctx, const pc2_key* key, int op, long* montmuls, long* montmuls_half, int* limbs) {
  if (!ctx || !key || !montmuls || !montmuls_half || !limbs) return PC2_EINVAL;
  *montmuls_half = 0;
  const int w = ctx->window;
  int rc = PC2_OK;
  auto fill = [&](auto tag) -> int {
    constexpr int Lh = decltype(tag)::value;
    if (op == 0) {
      auto P = cached<EncCrtParams<Lh>>(key, KIND_ENC_CRT, w, [&](EncCrtParams<Lh>& p) { return make_enc_crt<Lh>(*key, w, p); }, &rc);
      if (!P) return rc;
      if constexpr (lift_route<Lh, 1>()) {
        *montmuls = (long)P->lp.e2.montmuls + P->lq.e2.montmuls;
        *montmuls_half = (long)P->lp.e1.montmuls + P->lq.e1.montmuls;
      } else {
        *montmuls = (long)P->ep.montmuls + P->eq.montmuls;
      }
      *limbs = Lh;
    } else if (op == 1) {
      auto P = cached<EncPubParams<2 * Lh>>(key, KIND_ENC_PUB, w, [&](EncPubParams<2 * Lh>& p) { return make_enc_pub<2 * Lh>(*key, w, p); }, &rc);
      if (!P) return rc;
      *montmuls = (long)P->e.montmuls + 1;
      *limbs = 2 * Lh;
    } else if (op == 2) {
      auto P = cached<DecParams<Lh>>(key, KIND_DEC, w, [&](DecParams<Lh>& p) { return make_dec<Lh>(*key, w, p); }, &rc);
      if (!P) return rc;
      *montmuls = (long)P->ep.montmuls + P->eq.montmuls;
      *limbs = Lh;
    } else {
      return PC2_EINVAL;
    }
    return PC2_OK;
  };
  switch (key->Lh) {
    case 8: return fill(std::integral_constant<int, 8>());
    case 16: return fill(std::integral_constant<int, 16>());
    case 32: return fill(std::integral_constant<int, 32>());
    case 64: return fill(std::integral_constant<int, 64>());
    case 96: return fill(std::integral_constant<int, 96>());
    case 128: return fill(std::integral_constant<int, 128>());
    default: return PC2_EUNSUPPORTED;
  }
}

size_t pc2_tiled_words(size_t count, int limbs) { return (count + 31) / 32 * 32 * (size_t)limbs; }

int pc2_pack(pc2_ctx* ctx, const uint32_t* d_canon, size_t count, int limbs, uint32_t* d_tiled, pc2_stream_t stream) {
  if (!ctx || limbs <= 0 || limbs % 4 || (count && (!d_canon || !d_tiled))) return PC2_EINVAL;
  if (!count) return PC2_OK;
  return launch_pack(d_canon, count, limbs, d_tiled, ctx->sms, (cudaStream_t)stream);
}

int pc2_unpack(pc2_ctx* ctx, const uint32_t* d_tiled, size_t count, int limbs, uint32_t* d_canon, pc2_stream_t stream) {
  if (!ctx || limbs <= 0 || limbs % 4 || (count && (!d_canon || !d_tiled))) return PC2_EINVAL;
  if (!count) return PC2_OK;
  return launch_unpack(d_tiled, count, limbs, d_canon, ctx->sms, (cudaStream_t)stream);
}

static int encrypt_any(pc2_ctx* ctx, const pc2_key* key, const uint64_t* m64, const uint32_t* mw, size_t count,
                       uint64_t seed, uint32_t stream, uint64_t e0, uint32_t* d_ct, pc2_stream_t cs, bool force_pub) {
  if (!ctx || !key || !d_ct || (!m64 && !mw)) return count ? PC2_EINVAL : PC2_OK;
  if (!count) return PC2_OK;
  ctx->ev_recorded = false;  // set again only if this call runs on the tensor cores
  const cudaStream_t st = (cudaStream_t)cs;
  if (key->priv && !force_pub) {
#define PC2_CALL_CRT(L) enc_crt<L>(ctx, key, m64, mw, count, seed, stream, e0, d_ct, st)
    PC2_DISPATCH_H(key->Lh, PC2_CALL_CRT)
  }
#define PC2_CALL_PUB(L) enc_pub<2 * L>(ctx, key, m64, mw, count, seed, stream, e0, d_ct, st)
  PC2_DISPATCH_H(key->Lh, PC2_CALL_PUB)
}

int pc2_encrypt(pc2_ctx* ctx, const pc2_key* key, const uint64_t* d_m, size_t count, uint64_t seed, uint32_t stream,
                uint64_t e0, uint32_t* d_ct, pc2_stream_t cstream) {
  if (count && !d_m) return PC2_EINVAL;
  return encrypt_any(ctx, key, d_m, nullptr, count, seed, stream, e0, d_ct, cstream, false);
}

int pc2_encrypt_wide(pc2_ctx* ctx, const pc2_key* key, const uint32_t* d_m, size_t count, uint64_t seed,
                     uint32_t stream, uint64_t e0, uint32_t* d_ct, pc2_stream_t cstream) {
  if (count && !d_m) return PC2_EINVAL;
  return encrypt_any(ctx, key, nullptr, d_m, count, seed, stream, e0, d_ct, cstream, false);
}

int pc2_encrypt_public(pc2_ctx* ctx, const pc2_key* key, const uint64_t* d_m, size_t count, uint64_t seed,
                       uint32_t stream, uint64_t e0, uint32_t* d_ct, pc2_stream_t cstream) {
  if (count && !d_m) return PC2_EINVAL;
  return encrypt_any(ctx, key, d_m, nullptr, count, seed, stream, e0, d_ct, cstream, true);
}

int pc2_decrypt(pc2_ctx* ctx, const pc2_key* key, const uint32_t* d_ct, size_t count, uint32_t* d_m,
                pc2_stream_t cstream) {
  if (!ctx || !key) return PC2_EINVAL;
  if (!key->priv) return PC2_EKEY;
  if (!count) return PC2_OK;
  if (!d_ct || !d_m) return PC2_EINVAL;
  ctx->ev_recorded = false;  // set again only if this call runs on the tensor cores
  const cudaStream_t st = (cudaStream_t)cstream;
#define PC2_CALL_DEC(L) dec<L>(ctx, key, d_ct, count, d_m, st)
  PC2_DISPATCH_H(key->Lh, PC2_CALL_DEC)
}

int pc2_hom_sum(pc2_ctx* ctx, const pc2_key* key, const uint32_t* d_ct, size_t groups, size_t count, uint32_t* d_out,
                pc2_stream_t cstream) {
  if (!ctx || !key || groups == 0) return PC2_EINVAL;
  if (!count) return PC2_OK;
  if (!d_ct || !d_out) return PC2_EINVAL;
  std::unique_ptr<const uint32_t*[]> srcs(new (std::nothrow) const uint32_t*[groups]);
  if (!srcs) return PC2_ENOMEM;
  const size_t stride = pc2_tiled_words(count, 2 * key->Lh);
  for (size_t g = 0; g < groups; ++g) srcs[g] = d_ct + g * stride;
  const cudaStream_t st = (cudaStream_t)cstream;
#define PC2_CALL_SUM(L) hom_sum<2 * L>(ctx, key, srcs.get(), groups, count, d_out, st)
  PC2_DISPATCH_H(key->Lh, PC2_CALL_SUM)
}

int pc2_hom_add(pc2_ctx* ctx, const pc2_key* key, const uint32_t* d_a, const uint32_t* d_b, size_t count,
                uint32_t* d_out, pc2_stream_t cstream) {
  if (!ctx || !key) return PC2_EINVAL;
  if (!count) return PC2_OK;
  if (!d_a || !d_b || !d_out) return PC2_EINVAL;
  const uint32_t* srcs[2] = {d_a, d_b};
  const cudaStream_t st = (cudaStream_t)cstream;
#define PC2_CALL_ADD(L) hom_sum<2 * L>(ctx, key, srcs, 2, count, d_out, st)
  PC2_DISPATCH_H(key->Lh, PC2_CALL_ADD)
}

int pc2_hom_scal(pc2_ctx* ctx, const pc2_key* key, const uint32_t* d_ct, const uint64_t* d_k, size_t count,
                 uint32_t* d_out, pc2_stream_t cstream) {
  if (!ctx || !key) return PC2_EINVAL;
  if (!count) return PC2_OK;
  if (!d_ct || !d_k || !d_out) return PC2_EINVAL;
  const cudaStream_t st = (cudaStream_t)cstream;
#define PC2_CALL_SCAL(L) hom_scal<2 * L>(ctx, key, d_ct, d_k, count, d_out, st)
  PC2_DISPATCH_H(key->Lh, PC2_CALL_SCAL)
}

int pc2_hom_scal_wide(pc2_ctx* ctx, const pc2_key* key, const uint32_t* d_ct, const uint32_t* d_k, size_t count,
                      uint32_t* d_out, pc2_stream_t cstream) {
  if (!ctx || !key) return PC2_EINVAL;
  if (!count) return PC2_OK;
  if (!d_ct || !d_k || !d_out) return PC2_EINVAL;
  const cudaStream_t st = (cudaStream_t)cstream;
#define PC2_CALL_SCALW(L) hom_scal_wide<2 * L>(ctx, key, d_ct, d_k, count, d_out, st)
  PC2_DISPATCH_H(key->Lh, PC2_CALL_SCALW)
}

}  // extern "C"
