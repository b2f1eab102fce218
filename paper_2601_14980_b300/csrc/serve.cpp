// serve.cpp -- the serving form: a request loop on one GPU.
//
// Callers submit encrypt, decrypt and aggregate requests (host buffers) from
// any thread; a worker thread owns the GPU side:
//   admission  a request is admitted when its input and output buffers fit
//              in the device arena (first fit, FIFO order, at most
//              max_active requests); its input is copied in on a copy stream;
//   steps      each step is one persistent launch (k_serve_step) over work
//              items taken from every admitted request in admission order,
//              up to a work budget per CTA; two steps are in flight on two
//              streams, so a step's CTAs start as the previous step's CTAs
//              retire and requests admitted meanwhile join the next step;
//   completion when a request's last item has run, its output is copied to
//              the caller's buffer and its arena space is freed.
// Mode 1 (the plain per-request path) runs the admitted requests one at a
// time through pc2_encrypt / pc2_decrypt / pc2_hom_sum instead.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/pc2.h"
#include "ctx.hpp"
#include "keys.hpp"
#include "pc2_kernels.h"
#include "pc2_serve.h"

namespace {

using Clock = std::chrono::steady_clock;

double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

// First-fit allocator over one device region (offsets in bytes, 256-byte aligned).
class Arena {
 public:
  void init(size_t cap) {
    cap_ = cap;
    free_.clear();
    if (cap) free_[0] = cap;
    used_ = peak_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) / 256 * 256;
    if (!bytes) bytes = 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, o = it->first;
        free_.erase(it);
        if (rest) free_[o + bytes] = rest;
        used_ += bytes;
        peak_ = std::max(peak_, used_);
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    if (!bytes) bytes = 256;
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  static size_t rounded(size_t bytes) { return bytes ? (bytes + 255) / 256 * 256 : 256; }
  size_t cap() const { return cap_; }
  size_t peak() const { return peak_; }

 private:
  size_t cap_ = 0, used_ = 0, peak_ = 0;
  std::map<size_t, size_t> free_;
};

struct Req {
  uint64_t ticket = 0;
  int op = 0;
  size_t count = 0;
  int groups = 1;
  uint64_t seed = 0, e0 = 0;
  uint32_t stream = 0;
  const void* h_in = nullptr;
  void* h_out = nullptr;
  size_t in_bytes = 0, out_bytes = 0, ct_stride = 0;
  size_t h_stride = 0;      // aggregate: words between the group arrays in h_in
  size_t in_off = 0, out_off = 0;
  size_t cursor = 0;        // next element to schedule
  size_t outstanding = 0;   // scheduled items not yet finished
  bool small = false;
  cudaEvent_t h2d = nullptr, d2h = nullptr;
  bool waited[2] = {false, false};
  int state = 0;            // 0 waiting, 1 active, 2 copying out, 3 done
  int rc = PC2_OK;
  double t_submit = 0, t_done = 0;
};

struct Slot {
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  pc2::ServeReq* d_reqs = nullptr;
  pc2::ServeItem* d_items = nullptr;
  uint32_t* d_next = nullptr;
  pc2::ServeReq* h_reqs = nullptr;   // pinned staging
  pc2::ServeItem* h_items = nullptr;
  size_t cap_reqs = 0, cap_items = 0;
  bool busy = false;
  std::vector<std::pair<std::shared_ptr<Req>, size_t>> owners;
};

}  // namespace

struct pc2_server {
  pc2_ctx* ctx = nullptr;
  const pc2_key* key = nullptr;
  int Lh = 0, mode = 0, max_active = 256;
  size_t small_request = 4096;
  double step_budget = 1.0;
  unsigned char* arena_mem = nullptr;
  Arena arena;
  void* d_key = nullptr;
  void* d_const = nullptr;
  int tabw = 0, grid = 0;
  size_t cta_words = 0, smem = 0;
  uint32_t* scratch = nullptr;  // one region of grid x cta_words words per step slot
  Slot slots[2];
  cudaStream_t copy_in = nullptr, copy_out = nullptr;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  int failed = PC2_OK;
  std::deque<std::shared_ptr<Req>> waiting;
  std::vector<std::shared_ptr<Req>> active;
  std::unordered_map<uint64_t, std::shared_ptr<Req>> tickets;
  uint64_t next_ticket = 1;
  uint64_t completed = 0, steps = 0, items = 0;
};

namespace pc2 {

template <int Lh>
static int serve_setup(pc2_server* S) {
  std::unique_ptr<ServeKey<Lh>> K(new (std::nothrow) ServeKey<Lh>);
  if (!K) return PC2_ENOMEM;
  std::memset(K.get(), 0, sizeof(ServeKey<Lh>));
  int rc = make_enc_crt<Lh>(*S->key, S->ctx->window, K->enc);
  if (rc) return rc;
  if ((rc = make_dec<Lh>(*S->key, S->ctx->window, K->dec))) return rc;
  fill_mod(K->n2, S->key->n2);
  {
    const Mont M(S->key->n2, 2 * Lh);
    Big r = Big(1);
    for (int g = 0; g <= kMaxGroups; ++g) {
      r.to_words(K->rpow[g], 2 * Lh);
      r = mulmod(r, M.R1, S->key->n2);
    }
  }
  ServeConst<Lh> C;
  std::memcpy(C.mp, K->enc.mp.n, sizeof(C.mp));
  std::memcpy(C.mq, K->enc.mq.n, sizeof(C.mq));
  std::memcpy(C.n2, K->n2.n, sizeof(C.n2));
  std::memcpy(C.hp, K->enc.lp.h.n, sizeof(C.hp));
  std::memcpy(C.hq, K->enc.lq.h.n, sizeof(C.hq));
  if (cudaMalloc(&S->d_key, sizeof(ServeKey<Lh>)) != cudaSuccess || cudaMalloc(&S->d_const, sizeof(C)) != cudaSuccess)
    return PC2_ENOMEM;
  if (cudaMemcpy(S->d_key, K.get(), sizeof(ServeKey<Lh>), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(S->d_const, &C, sizeof(C), cudaMemcpyHostToDevice) != cudaSuccess)
    return PC2_ECUDA;
  const int w = std::max(std::max(K->enc.ep.w, K->enc.eq.w), std::max(K->dec.ep.w, K->dec.eq.w));
  S->tabw = (1 << (w - 1)) * Lh;
  S->cta_words = (size_t)kThreads * ((size_t)S->tabw + 8 * (size_t)(2 * Lh + 4));
  S->smem = (size_t)4 * std::max((size_t)Lh * kThreads, (size_t)2 * Lh * (kThreads / serve_agg_lanes(2 * Lh)));
  const int per = serve_blocks_per_sm<Lh>(S->smem);
  if (per < 1) return PC2_ECUDA;
  S->grid = per * S->ctx->sms;
  if (cudaMalloc(&S->scratch, 2 * S->cta_words * (size_t)S->grid * 4) != cudaSuccess) return PC2_ENOMEM;
  return PC2_OK;
}

// The server whose key is in constant memory, per key size (one constant
// block per size in the process); a step of another server copies its own
// key in first (all steps of the process then see it, so two servers of one
// key size must not run steps at the same time).
static std::mutex g_const_mu;
static const pc2_server* g_const_owner[2] = {nullptr, nullptr};

static int launch_step(pc2_server* S, const ServeParams& P, Slot& sl, bool one_lane_split) {
  {
    std::lock_guard<std::mutex> g(g_const_mu);
    const pc2_server*& own = g_const_owner[S->Lh == 16 ? 0 : 1];
    if (own != S) {
      const int rc = S->Lh == 16 ? serve_set_const<16>(static_cast<const ServeConst<16>*>(S->d_const), sl.st)
                                 : serve_set_const<64>(static_cast<const ServeConst<64>*>(S->d_const), sl.st);
      if (rc) return rc;
      own = S;
    }
  }
  if (S->Lh == 16) return launch_serve_step<16>(P, S->smem, S->grid, sl.st, one_lane_split);
  return launch_serve_step<64>(P, S->smem, S->grid, sl.st, one_lane_split);
}

// Relative duration of one work item (one-lane encryption item = 1).
static double item_cost(int kind, int groups) {
  switch (kind) {
    case SK_ENC1: return 1.0;
    case SK_ENC1S: return 0.5;
    case SK_ENC2: return 0.3;
    case SK_ENC8: return 0.1;
    case SK_DEC1: return 0.5;
    case SK_DEC1S: return 0.25;
    case SK_DEC2: return 0.15;
    case SK_DEC8: return 0.05;
    default: return 0.002 * groups;
  }
}

static bool ensure_slot_cap(Slot& sl, size_t nreq, size_t nitem) {
  if (nreq > sl.cap_reqs) {
    if (sl.d_reqs) cudaFree(sl.d_reqs);
    if (sl.h_reqs) cudaFreeHost(sl.h_reqs);
    sl.d_reqs = nullptr;
    sl.h_reqs = nullptr;
    sl.cap_reqs = 0;
    if (cudaMalloc(&sl.d_reqs, nreq * sizeof(ServeReq)) != cudaSuccess ||
        cudaMallocHost(&sl.h_reqs, nreq * sizeof(ServeReq)) != cudaSuccess)
      return false;
    sl.cap_reqs = nreq;
  }
  if (nitem > sl.cap_items) {
    if (sl.d_items) cudaFree(sl.d_items);
    if (sl.h_items) cudaFreeHost(sl.h_items);
    sl.d_items = nullptr;
    sl.h_items = nullptr;
    sl.cap_items = 0;
    if (cudaMalloc(&sl.d_items, nitem * sizeof(ServeItem)) != cudaSuccess ||
        cudaMallocHost(&sl.h_items, nitem * sizeof(ServeItem)) != cudaSuccess)
      return false;
    sl.cap_items = nitem;
  }
  return true;
}

// Builds and launches one step in slot `si`; false when there is nothing to run.
static int build_step(pc2_server* S, int si, bool* launched) {
  *launched = false;
  Slot& sl = S->slots[si];
  std::vector<ServeReq> reqs;
  std::vector<ServeItem> its;
  std::vector<std::pair<std::shared_ptr<Req>, size_t>> owners;
  double budget = S->step_budget * S->grid;
  const int L2 = 2 * S->Lh;
  // Lanes per element for each request of this step: start every request at
  // 8 lanes per CRT half (16 per element) and, while the step's threads do
  // not fit one resident wave, move the request with the largest demand down
  // to 2 lanes per half, 1 lane per half, then one lane per element; small
  // requests keep the 16.
  static const int kLaneSteps[4] = {2 * kServeLanesSmall, 4, 2, 1};
  std::vector<int> lvl(S->active.size(), 0);
  {
    const double cap = (double)S->grid * kThreads;
    auto demand = [&](size_t i) {
      const auto& r = S->active[i];
      if (r->state != 1 || r->op == SERVE_AGGREGATE || r->cursor >= r->count) return 0.0;
      return (double)(r->count - r->cursor) * kLaneSteps[lvl[i]];
    };
    double total = 0;
    for (size_t i = 0; i < lvl.size(); ++i) total += demand(i);
    while (total > cap) {
      size_t arg = lvl.size();
      double worst = 0;
      for (size_t i = 0; i < lvl.size(); ++i) {
        if (lvl[i] == 3 || S->active[i]->small) continue;
        const double d = demand(i);
        if (d > worst) {
          worst = d;
          arg = i;
        }
      }
      if (arg == lvl.size()) break;
      total -= worst;
      ++lvl[arg];
      total += demand(arg);
    }
  }
  for (size_t ai = 0; ai < S->active.size(); ++ai) {
    auto& r = S->active[ai];
    if (budget <= 0) break;
    if (r->state != 1 || r->cursor >= r->count) continue;
    const uint32_t ri = (uint32_t)reqs.size();
    ServeReq d;
    std::memset(&d, 0, sizeof(d));
    unsigned char* base = S->arena_mem;
    d.m64 = reinterpret_cast<const uint64_t*>(base + r->in_off);
    d.ct_in = reinterpret_cast<const uint32_t*>(base + r->in_off);
    d.out = reinterpret_cast<uint32_t*>(base + r->out_off);
    d.count = r->count;
    d.ct_stride = r->ct_stride;
    d.seed = r->seed;
    d.e0 = r->e0;
    d.stream = r->stream;
    d.op = (uint32_t)r->op;
    d.groups = (uint32_t)r->groups;
    reqs.push_back(d);
    if (!r->waited[si]) {
      if (cudaStreamWaitEvent(sl.st, r->h2d, 0) != cudaSuccess) return PC2_ECUDA;
      r->waited[si] = true;
    }
    int kind;
    uint32_t per;
    if (r->op == SERVE_AGGREGATE) {
      kind = SK_AGG;
      per = (uint32_t)(kThreads / serve_agg_lanes(L2));
    } else if (lvl[ai] == 0 || r->small) {
      kind = r->op == SERVE_ENCRYPT ? SK_ENC8 : SK_DEC8;
      per = kThreads / kServeLanesSmall / 2;  // two lane groups (the CRT halves) per element
    } else if (lvl[ai] == 1) {
      kind = r->op == SERVE_ENCRYPT ? SK_ENC2 : SK_DEC2;
      per = kThreads / 2 / 2;
    } else if (lvl[ai] == 2) {
      kind = r->op == SERVE_ENCRYPT ? SK_ENC1S : SK_DEC1S;
      per = kThreads / 2;
    } else {
      kind = r->op == SERVE_ENCRYPT ? SK_ENC1 : SK_DEC1;
      per = kThreads;
    }
    size_t n_items = 0;
    while (r->cursor < r->count && budget > 0) {
      const uint32_t n = (uint32_t)std::min<size_t>(per, r->count - r->cursor);
      its.push_back(ServeItem{ri, (uint32_t)r->cursor, n, (uint32_t)kind});
      r->cursor += n;
      budget -= item_cost(kind, r->groups);
      ++n_items;
    }
    r->outstanding += n_items;
    owners.emplace_back(r, n_items);
  }
  if (its.empty()) return PC2_OK;
  // one-lane-per-half items run in their own kernel, after the others
  const size_t n_main = (size_t)(std::stable_partition(its.begin(), its.end(),
                                                       [](const ServeItem& x) {
                                                         return x.kind != SK_ENC1S && x.kind != SK_DEC1S;
                                                       }) -
                                 its.begin());
  if (!ensure_slot_cap(sl, reqs.size(), its.size())) return PC2_ENOMEM;
  std::memcpy(sl.h_reqs, reqs.data(), reqs.size() * sizeof(ServeReq));
  std::memcpy(sl.h_items, its.data(), its.size() * sizeof(ServeItem));
  if (cudaMemcpyAsync(sl.d_reqs, sl.h_reqs, reqs.size() * sizeof(ServeReq), cudaMemcpyHostToDevice, sl.st) ||
      cudaMemcpyAsync(sl.d_items, sl.h_items, its.size() * sizeof(ServeItem), cudaMemcpyHostToDevice, sl.st) ||
      cudaMemsetAsync(sl.d_next, 0, 8, sl.st))
    return PC2_ECUDA;
  ServeParams P;
  std::memset(&P, 0, sizeof(P));
  P.key = S->d_key;
  P.reqs = sl.d_reqs;
  P.items = sl.d_items;
  P.nitems = (uint32_t)its.size();
  P.tabw = S->tabw;
  P.next = sl.d_next;
  // each slot has its own scratch: the two steps' CTAs run at the same time
  P.scratch = S->scratch + (size_t)si * S->grid * S->cta_words;
  P.cta_words = S->cta_words;
  P.status = S->ctx->status;
  int rc = PC2_OK;
  if (n_main) {
    P.nitems = (uint32_t)n_main;
    rc = launch_step(S, P, sl, false);
    if (rc) return rc;
  }
  if (n_main < its.size()) {
    P.items = sl.d_items + n_main;
    P.nitems = (uint32_t)(its.size() - n_main);
    P.next = sl.d_next + 1;
    rc = launch_step(S, P, sl, true);
    if (rc) return rc;
  }
  if (cudaEventRecord(sl.ev, sl.st) != cudaSuccess) return PC2_ECUDA;
  sl.owners = std::move(owners);
  sl.busy = true;
  ++S->steps;
  S->items += its.size();
  *launched = true;
  return PC2_OK;
}

static int plain_run(pc2_server* S, Req& r) {
  unsigned char* base = S->arena_mem;
  const cudaStream_t st = S->slots[0].st;
  if (cudaStreamWaitEvent(st, r.h2d, 0) != cudaSuccess) return PC2_ECUDA;
  int rc;
  if (r.op == SERVE_ENCRYPT)
    rc = pc2_encrypt(S->ctx, S->key, reinterpret_cast<const uint64_t*>(base + r.in_off), r.count, r.seed, r.stream,
                     r.e0, reinterpret_cast<uint32_t*>(base + r.out_off), (pc2_stream_t)st);
  else if (r.op == SERVE_DECRYPT)
    rc = pc2_decrypt(S->ctx, S->key, reinterpret_cast<const uint32_t*>(base + r.in_off), r.count,
                     reinterpret_cast<uint32_t*>(base + r.out_off), (pc2_stream_t)st);
  else
    rc = pc2_hom_sum(S->ctx, S->key, reinterpret_cast<const uint32_t*>(base + r.in_off), (size_t)r.groups, r.count,
                     reinterpret_cast<uint32_t*>(base + r.out_off), (pc2_stream_t)st);
  if (rc) return rc;
  if (cudaEventRecord(S->slots[0].ev, st) != cudaSuccess) return PC2_ECUDA;
  if (cudaStreamWaitEvent(S->copy_out, S->slots[0].ev, 0) != cudaSuccess) return PC2_ECUDA;
  return PC2_OK;
}

static void fail_all(pc2_server* S, int rc) {
  std::lock_guard<std::mutex> g(S->mu);
  S->failed = rc;
  for (auto& r : S->active) {
    r->rc = rc;
    r->state = 3;
    r->t_done = now_s();
  }
  for (auto& r : S->waiting) {
    r->rc = rc;
    r->state = 3;
    r->t_done = now_s();
  }
  S->active.clear();
  S->waiting.clear();
  S->cv_done.notify_all();
}

static void worker_main(pc2_server* S) {
  cudaSetDevice(S->ctx->device);
  for (;;) {
    bool progress = false;
    // 1. retire finished steps
    for (auto& sl : S->slots) {
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.ev);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) return fail_all(S, PC2_ECUDA);
      for (auto& o : sl.owners) o.first->outstanding -= o.second;
      sl.owners.clear();
      sl.busy = false;
      progress = true;
    }
    std::vector<std::shared_ptr<Req>> finished;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->stop && S->waiting.empty() && S->active.empty()) break;
      // 2. outputs of fully computed requests
      for (auto& r : S->active) {
        if (r->state == 1 && r->cursor >= r->count && r->outstanding == 0 && S->mode == 0) {
          if (cudaMemcpyAsync(r->h_out, S->arena_mem + r->out_off, r->out_bytes, cudaMemcpyDeviceToHost,
                              S->copy_out) != cudaSuccess ||
              cudaEventRecord(r->d2h, S->copy_out) != cudaSuccess) {
            lk.unlock();
            return fail_all(S, PC2_ECUDA);
          }
          r->state = 2;
          progress = true;
        }
      }
      // 3. finished copies
      for (auto it = S->active.begin(); it != S->active.end();) {
        auto& r = *it;
        if (r->state == 2) {
          const cudaError_t q = cudaEventQuery(r->d2h);
          if (q == cudaSuccess) {
            r->state = 3;
            r->t_done = now_s();
            S->arena.release(r->in_off, r->in_bytes);
            S->arena.release(r->out_off, r->out_bytes);
            ++S->completed;
            finished.push_back(r);
            it = S->active.erase(it);
            progress = true;
            continue;
          }
          if (q != cudaErrorNotReady) {
            lk.unlock();
            return fail_all(S, PC2_ECUDA);
          }
        }
        ++it;
      }
      if (!finished.empty()) S->cv_done.notify_all();
      // 4. admission (FIFO, by memory)
      while (!S->waiting.empty() && (int)S->active.size() < S->max_active) {
        auto& r = S->waiting.front();
        size_t io = 0, oo = 0;
        if (!S->arena.alloc(r->in_bytes, &io)) break;
        if (!S->arena.alloc(r->out_bytes, &oo)) {
          S->arena.release(io, r->in_bytes);
          break;
        }
        r->in_off = io;
        r->out_off = oo;
        // inputs in; aggregate operands packed group by group (ct_stride words apart)
        bool ok = true;
        if (r->op == PC2_OP_AGGREGATE) {
          for (int gi = 0; gi < r->groups && ok; ++gi)
            ok = cudaMemcpyAsync(S->arena_mem + io + (size_t)gi * r->ct_stride * 4,
                                 static_cast<const uint32_t*>(r->h_in) + (size_t)gi * r->h_stride, r->ct_stride * 4,
                                 cudaMemcpyHostToDevice, S->copy_in) == cudaSuccess;
        } else {
          ok = cudaMemcpyAsync(S->arena_mem + io, r->h_in, r->in_bytes, cudaMemcpyHostToDevice, S->copy_in) ==
               cudaSuccess;
        }
        if (!ok || cudaEventRecord(r->h2d, S->copy_in) != cudaSuccess) {
          lk.unlock();
          return fail_all(S, PC2_ECUDA);
        }
        r->state = 1;
        S->active.push_back(r);
        S->waiting.pop_front();
        progress = true;
      }
    }
    // 5. work
    if (S->mode == 0) {
      for (int si = 0; si < 2; ++si) {
        if (S->slots[si].busy) continue;
        bool launched = false;
        std::unique_lock<std::mutex> lk(S->mu);
        const int rc = build_step(S, si, &launched);
        lk.unlock();
        if (rc) return fail_all(S, rc);
        progress = progress || launched;
        if (!launched) break;
      }
    } else {
      // plain path: the oldest admitted request, alone
      std::shared_ptr<Req> r;
      {
        std::lock_guard<std::mutex> g(S->mu);
        for (auto& a : S->active)
          if (a->state == 1) {
            r = a;
            break;
          }
      }
      if (r) {
        const int rc = plain_run(S, *r);
        if (rc) return fail_all(S, rc);
        if (cudaMemcpyAsync(r->h_out, S->arena_mem + r->out_off, r->out_bytes, cudaMemcpyDeviceToHost,
                            S->copy_out) != cudaSuccess ||
            cudaEventRecord(r->d2h, S->copy_out) != cudaSuccess || cudaEventSynchronize(r->d2h) != cudaSuccess)
          return fail_all(S, PC2_ECUDA);
        std::lock_guard<std::mutex> g(S->mu);
        r->cursor = r->count;
        r->state = 2;  // step 3 of the next pass retires it
        progress = true;
      }
    }
    if (!progress) {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait_for(lk, std::chrono::microseconds(100));
    }
  }
}

}  // namespace pc2

using namespace pc2;

extern "C" {

int pc2_server_create(pc2_ctx* ctx, const pc2_key* key, const pc2_server_params* prm, pc2_server** out) {
  if (!ctx || !key || !prm || !out || !prm->arena_bytes || prm->mode < 0 || prm->mode > 1) return PC2_EINVAL;
  if (!key->priv) return PC2_EKEY;
  if (key->Lh != 16 && key->Lh != 64) return PC2_EUNSUPPORTED;
  *out = nullptr;
  std::unique_ptr<pc2_server> S(new (std::nothrow) pc2_server);
  if (!S) return PC2_ENOMEM;
  S->ctx = ctx;
  S->key = key;
  S->Lh = key->Lh;
  S->mode = prm->mode;
  if (prm->max_active > 0) S->max_active = prm->max_active;
  if (prm->small_request > 0) S->small_request = prm->small_request;
  if (prm->step_budget > 0) S->step_budget = prm->step_budget;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return PC2_ECUDA;
  int rc = key->Lh == 16 ? serve_setup<16>(S.get()) : serve_setup<64>(S.get());
  if (rc) return rc;
  if (cudaMalloc(&S->arena_mem, prm->arena_bytes) != cudaSuccess) return PC2_ENOMEM;
  S->arena.init(prm->arena_bytes);
  for (auto& sl : S->slots) {
    if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&sl.d_next, 8) != cudaSuccess)
      return PC2_ECUDA;
  }
  if (cudaStreamCreateWithFlags(&S->copy_in, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&S->copy_out, cudaStreamNonBlocking) != cudaSuccess)
    return PC2_ECUDA;
  S->worker = std::thread(worker_main, S.get());
  *out = S.release();
  return PC2_OK;
}

void pc2_server_destroy(pc2_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> g(g_const_mu);
    for (auto& o : g_const_owner)
      if (o == S) o = nullptr;
  }
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  cudaSetDevice(S->ctx->device);
  cudaDeviceSynchronize();
  for (auto& sl : S->slots) {
    if (sl.st) cudaStreamDestroy(sl.st);
    if (sl.ev) cudaEventDestroy(sl.ev);
    if (sl.d_next) cudaFree(sl.d_next);
    if (sl.d_reqs) cudaFree(sl.d_reqs);
    if (sl.d_items) cudaFree(sl.d_items);
    if (sl.h_reqs) cudaFreeHost(sl.h_reqs);
    if (sl.h_items) cudaFreeHost(sl.h_items);
  }
  for (auto& kv : S->tickets) {
    if (kv.second->h2d) cudaEventDestroy(kv.second->h2d);
    if (kv.second->d2h) cudaEventDestroy(kv.second->d2h);
  }
  if (S->copy_in) cudaStreamDestroy(S->copy_in);
  if (S->copy_out) cudaStreamDestroy(S->copy_out);
  if (S->arena_mem) cudaFree(S->arena_mem);
  if (S->scratch) cudaFree(S->scratch);
  if (S->d_key) cudaFree(S->d_key);
  if (S->d_const) cudaFree(S->d_const);
  delete S;
}

int pc2_server_submit(pc2_server* S, int op, const void* h_in, size_t count, int groups, size_t h_stride,
                      uint64_t seed, uint32_t stream, uint64_t e0, void* h_out, uint64_t* ticket) {
  if (!S || !h_in || !h_out || !ticket || !count || op < PC2_OP_ENCRYPT || op > PC2_OP_AGGREGATE) return PC2_EINVAL;
  if (op == PC2_OP_AGGREGATE && (groups < 2 || groups > kMaxGroups)) return PC2_EINVAL;
  auto r = std::make_shared<Req>();
  r->op = op;
  r->count = count;
  r->groups = op == PC2_OP_AGGREGATE ? groups : 1;
  r->seed = seed;
  r->stream = stream;
  r->e0 = e0;
  r->h_in = h_in;
  r->h_out = h_out;
  const int L2 = 2 * S->Lh;
  r->ct_stride = pc2_tiled_words(count, L2);
  r->h_stride = h_stride ? h_stride : r->ct_stride;
  if (op == PC2_OP_AGGREGATE && r->h_stride < r->ct_stride) return PC2_EINVAL;
  if (op == PC2_OP_ENCRYPT) {
    r->in_bytes = count * 8;
    r->out_bytes = r->ct_stride * 4;
  } else if (op == PC2_OP_DECRYPT) {
    r->in_bytes = r->ct_stride * 4;
    r->out_bytes = pc2_tiled_words(count, S->Lh) * 4;
  } else {
    r->in_bytes = (size_t)groups * r->ct_stride * 4;
    r->out_bytes = r->ct_stride * 4;
  }
  if (Arena::rounded(r->in_bytes) + Arena::rounded(r->out_bytes) > S->arena.cap()) return PC2_ENOMEM;
  r->small = count <= S->small_request;
  if (cudaEventCreateWithFlags(&r->h2d, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&r->d2h, cudaEventDisableTiming) != cudaSuccess)
    return PC2_ECUDA;
  {
    std::lock_guard<std::mutex> g(S->mu);
    if (S->failed) return S->failed;
    if (S->stop) return PC2_EINVAL;
    r->ticket = S->next_ticket++;
    r->t_submit = now_s();
    S->waiting.push_back(r);
    S->tickets[r->ticket] = r;
    *ticket = r->ticket;
  }
  S->cv_work.notify_all();
  return PC2_OK;
}

int pc2_server_wait(pc2_server* S, uint64_t ticket, double timeout_s, double* latency_s) {
  if (!S) return PC2_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->tickets.find(ticket);
  if (it == S->tickets.end()) return PC2_EINVAL;
  auto r = it->second;
  const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
  while (r->state != 3) {
    if (S->cv_done.wait_until(lk, until) == std::cv_status::timeout && r->state != 3) return PC2_ETIMEOUT;
  }
  if (latency_s) *latency_s = r->t_done - r->t_submit;
  S->tickets.erase(it);
  lk.unlock();
  cudaEventDestroy(r->h2d);
  cudaEventDestroy(r->d2h);
  r->h2d = r->d2h = nullptr;
  return r->rc;
}

int pc2_server_stats(pc2_server* S, uint64_t* completed, uint64_t* steps, uint64_t* items, size_t* arena_peak) {
  if (!S) return PC2_EINVAL;
  std::lock_guard<std::mutex> g(S->mu);
  if (completed) *completed = S->completed;
  if (steps) *steps = S->steps;
  if (items) *items = S->items;
  if (arena_peak) *arena_peak = S->arena.peak();
  return PC2_OK;
}

}  // extern "C"
