// tc_paillier.cu -- key-owner encryption and CRT decryption at 2048-bit n
// with the full-width powers on the tensor-core Montgomery product
// (tc_core.cuh).
//
// Each operation runs as three launches:
//   pre   (integer pipe) the per-element set-up of both CRT halves: for
//         encryption the lifted route's half-width power
//         s = r^(h' mod (h-1)) mod h and its lift s R mod h^2; for decryption
//         c R mod h^2;
//   power (tensor cores) x <- x^E in the Montgomery domain mod h^2 for all
//         elements, E = h (encryption, r^n = s^h mod h^2) or h - 1
//         (decryption), by the same sliding-window schedule as the one-kernel
//         path; once for h = p, once for h = q;
//   post  (integer pipe) the rest of Eq. (itq1) per half (times g^m = 1 + m n)
//         and the recombination of Eq. (gA-C-B), or L_h and the Garner
//         recombination of the decryption.
// The results are the same integers as k_enc_crt / k_dec_crt.
#include <cuda_runtime.h>

#include <cstring>

#include "paillier_kernels.cuh"
#include "pc2_tc.h"
#include "tc_core.cuh"

namespace pc2 {

// ------------------------------------------------------------------ the power on the tensor cores
struct TcExpParams {
  tc::Mod m;
  Sched<kMaxSchedHalf> e;
};
static_assert(sizeof(TcExpParams) + 256 <= 32764, "parameter block too large");

// x <- x^E (Montgomery domain, 64 words, tiled, in place).  tabs: per CTA
// (2^(w-1) + 1) entries of 64 words x 128 elements (odd powers, then x^2).
__global__ void __launch_bounds__(tc::kThreads, 2)
    k_modexp_tc(const __grid_constant__ TcExpParams P, uint32_t* __restrict__ xy, size_t count,
                uint32_t* __restrict__ tabs, int* status) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const tc::Smem s = tc::smem_layout(smem);
  const uint32_t tmem = tc::setup(s, P.m);
  if ((threadIdx.x >> 5) == 4) {
    tc::serve(s, tmem);
  } else {
    constexpr int L = tc::kL;
    const int e = threadIdx.x;
    const int ntab = 1 << (P.e.w - 1);
    const size_t ts = tc::kTileE;  // words of one table entry are tc::kTileE apart
    uint32_t* tab = tabs + (size_t)blockIdx.x * (size_t)(ntab + 1) * L * tc::kTileE + e;
    auto entry = [&](int k) { return tab + (size_t)k * L * ts; };
    tc::State st{0u, true};
    const size_t ntiles = (count + tc::kTileE - 1) / tc::kTileE;
    const int idx0 = (int)(P.e.step[0] & 0xffu) - 1;
    for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      size_t g = tile * tc::kTileE + e;
      const bool valid = g < count;
      if (!valid) g = count - 1;
      uint32_t a[L];
#pragma unroll
      for (int j = 0; j < L; ++j) a[j] = xy[tiled_index(g, j, L)];
      {
        uint32_t* t0 = entry(0);
#pragma unroll
        for (int j = 0; j < L; ++j) t0[j * ts] = a[j];
      }
      // one product per trip: x^2, then the odd powers x^(2k+1) = x^(2k-1) x^2,
      // then the schedule's squarings and table multiplies
      int phase = ntab > 1 ? 0 : 2, k = 1, si = 1, q = 0;
      if (phase == 2) {
        const uint32_t* t = entry(idx0);
#pragma unroll
        for (int j = 0; j < L; ++j) a[j] = t[j * ts];
      }
      for (;;) {
        int src = -1;  // -1: a itself, else a table entry
        if (phase == 1) {
          src = ntab;
        } else if (phase == 2) {
          bool more = false;
          while (si < P.e.nsteps) {
            const uint32_t stp = P.e.step[si];
            const int nsq = (int)(stp >> 8), idx = (int)(stp & 0xffu) - 1;
            if (q < nsq) {
              ++q;
              more = true;
              break;
            }
            if (q == nsq && idx >= 0) {
              ++q;
              src = idx;
              more = true;
              break;
            }
            ++si;
            q = 0;
          }
          if (!more) break;
        }
        if (src < 0) {
          tc::montsqr(a, s, tmem, P.m.n, st);
        } else {
          tc::write_b_global(s, entry(src), ts);
          tc::montmul(a, s, tmem, P.m.n, st);
        }
        if (phase == 0) {  // x^2: keep it, restart from x
          uint32_t* t2 = entry(ntab);
          const uint32_t* t0 = entry(0);
#pragma unroll
          for (int j = 0; j < L; ++j) {
            t2[j * ts] = a[j];
            a[j] = t0[j * ts];
          }
          phase = 1;
        } else if (phase == 1) {
          uint32_t* tk = entry(k);
#pragma unroll
          for (int j = 0; j < L; ++j) tk[j * ts] = a[j];
          if (++k == ntab) {
            const uint32_t* t = entry(idx0);
#pragma unroll
            for (int j = 0; j < L; ++j) a[j] = t[j * ts];
            phase = 2;
          }
        }
      }
      if (valid) {
#pragma unroll
        for (int j = 0; j < L; ++j) xy[tiled_index(g, j, L)] = a[j];
      }
    }
    tc::stop(s);
    if (!st.ok && status) atomicOr(status, PC2_ST_TIMEOUT);
  }
  tc::teardown(tmem);
}

// ------------------------------------------------------------------ encryption: set-up and finish
// A = s R mod h^2 with s = r^(h' mod (h-1)) mod h from the raw draw X (the
// lifted route of LiftConst, up to its power by h).
template <int Lh>
__device__ __forceinline__ void lift_prep(const ModConst<Lh>& M, const LiftConst<Lh>& H, const Col& X, const Col& A,
                                          const Col& B, const Col& C, const Col& TT, const Col& tab, const Col& bsh,
                                          const Grp<1>& g) {
  constexpr int Lp = Lh / 2;
  g_to_mont_2l(A, X.off(Lp), H.h.n, H.h.r2, H.h.r3, H.h.np, Lp, B, C, TT);  // x1 R_h
  g_copy_param(B, H.h.r2, Lp);
  g_mont(A, A, B, H.h.n, H.h.np, Lp, TT);                                  // x1 R_h^2
  g_mont(C, X, B, H.h.n, H.h.np, Lp, TT);                                  // x0 R_h
  g_addmod(A, A, C, H.h.n, Lp);                                            // r R_h mod h
  __syncwarp();
  {
    uint32_t a[Lp];
    load_seg(a, A, g);
    run_modexp<Lp, 1>(a, H.e1, H.h.n, H.h.np, tab, bsh, g);              // s R_h
    store_seg(A, a, g);
  }
  __syncwarp();
  for (int j = Lp; j < Lh; ++j) A[j] = 0u;
  g_copy_param(B, H.lift, Lh);
  g_mont(A, A, B, M.n, M.np, Lh, TT);                                      // s R mod h^2
}

template <int Lh>
__global__ void __launch_bounds__(kThreads, min_blocks(Lh, 1))
    k_enc_tc_pre(const __grid_constant__ EncCrtParams<Lh> P, size_t count, uint32_t* __restrict__ sp,
                 uint32_t* __restrict__ sq, uint32_t* __restrict__ scratch, int tabw) {
  extern __shared__ uint32_t bsh_all[];
  const Grp<1> g;
  const Layout ly(1);
  const Col bsh{bsh_all + ly.gl, ly.G};
  const Col tab = ly.slot(scratch, 0);
  const int SW = 2 * Lh + 4;
  const Col X = ly.slot(scratch, tabw + 0 * SW), A = ly.slot(scratch, tabw + 1 * SW),
            B = ly.slot(scratch, tabw + 2 * SW), C = ly.slot(scratch, tabw + 3 * SW),
            TT = ly.slot(scratch, tabw + 4 * SW);
  for (size_t base = (size_t)blockIdx.x * ly.G; base < count; base += (size_t)ly.Gtot) {
    size_t e = base + ly.gl;
    const bool valid = e < count;
    if (!valid) e = count - 1;
    const uint32_t sid = P.round_ptr ? ((*P.round_ptr << 8) | P.kind) : P.stream;
    gen_r(X, P.seed, sid, P.e0 + e, Lh + 2, 2 * Lh);
    lift_prep<Lh>(P.mp, P.lp, X, A, B, C, TT, tab, bsh, g);
    if (valid)
      for (int j = 0; j < Lh; ++j) sp[tiled_index(e, j, Lh)] = A[j];
    lift_prep<Lh>(P.mq, P.lq, X, A, B, C, TT, tab, bsh, g);
    if (valid)
      for (int j = 0; j < Lh; ++j) sq[tiled_index(e, j, Lh)] = A[j];
    __syncwarp();
  }
}

template <int Lh>
__global__ void __launch_bounds__(kThreads, min_blocks(Lh, 1))
    k_enc_tc_post(const __grid_constant__ EncCrtParams<Lh> P, const uint64_t* __restrict__ m64,
                  const uint32_t* __restrict__ mwide, size_t count, const uint32_t* __restrict__ yp,
                  const uint32_t* __restrict__ yq, uint32_t* __restrict__ out, uint32_t* __restrict__ scratch,
                  int* status, size_t base_out) {
  const Layout ly(1);
  const int SW = 2 * Lh + 4;
  const Col X = ly.slot(scratch, 0 * SW), GM = ly.slot(scratch, 1 * SW), A = ly.slot(scratch, 2 * SW),
            B = ly.slot(scratch, 3 * SW), C = ly.slot(scratch, 4 * SW), TT = ly.slot(scratch, 5 * SW),
            CP = ly.slot(scratch, 6 * SW), CQ = ly.slot(scratch, 7 * SW);
  for (size_t base = (size_t)blockIdx.x * ly.G; base < count; base += (size_t)ly.Gtot) {
    size_t e = base + ly.gl;
    const bool valid = e < count;
    if (!valid) e = count - 1;
    make_gm(GM, A, m64, mwide, e, P.nwords, Lh, 2 * Lh, valid, status);
    for (int h = 0; h < 2; ++h) {
      const ModConst<Lh>& M = h ? P.mq : P.mp;
      const uint32_t* y = h ? yq : yp;
      const Col& OUT = h ? CQ : CP;
      for (int j = 0; j < Lh; ++j) A[j] = y[tiled_index(e, j, Lh)];     // (r^n mod h^2) R
      g_to_mont_2l(B, GM, M.n, M.r2, M.r3, M.np, Lh, C, OUT, TT);      // (1 + m n) R mod h^2
      g_mont(C, A, B, M.n, M.np, Lh, TT);                               // c_h R
      g_zero(B, Lh);
      B[0] = 1u;
      g_mont(OUT, C, B, M.n, M.np, Lh, TT);                             // c_h
    }
    // Eq. (gA-C-B): c = c_p + [(c_q - c_p) (p^2)^-1 mod q^2] p^2  (c_p < p^2 < q^2)
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
    if (valid) write_tiled<1>(out, base_out + e, X, 2 * Lh, Grp<1>());
  }
}

// ------------------------------------------------------------------ decryption: set-up and finish
template <int Lh>
__global__ void __launch_bounds__(kThreads, min_blocks(Lh, 1))
    k_dec_tc_pre(const __grid_constant__ DecParams<Lh> P, const uint32_t* __restrict__ ct, size_t count,
                 uint32_t* __restrict__ sp, uint32_t* __restrict__ sq, uint32_t* __restrict__ scratch,
                 size_t ebase) {
  const Layout ly(1);
  const int SW = 2 * Lh + 4;
  const Col X = ly.slot(scratch, 0 * SW), A = ly.slot(scratch, 1 * SW), B = ly.slot(scratch, 2 * SW),
            C = ly.slot(scratch, 3 * SW), TT = ly.slot(scratch, 4 * SW);
  for (size_t base = (size_t)blockIdx.x * ly.G; base < count; base += (size_t)ly.Gtot) {
    size_t e = base + ly.gl;
    const bool valid = e < count;
    if (!valid) e = count - 1;
    for (int j = 0; j < 2 * Lh; ++j) X[j] = ct[tiled_index(ebase + e, j, 2 * Lh)];
    for (int h = 0; h < 2; ++h) {
      const ModConst<Lh>& M = h ? P.mq : P.mp;
      g_to_mont_2l(A, X, M.n, M.r2, M.r3, M.np, Lh, B, C, TT);  // c R mod h^2
      uint32_t* s = h ? sq : sp;
      if (valid)
        for (int j = 0; j < Lh; ++j) s[tiled_index(e, j, Lh)] = A[j];
    }
  }
}

template <int Lh>
__global__ void __launch_bounds__(kThreads, min_blocks(Lh, 1))
    k_dec_tc_post(const __grid_constant__ DecParams<Lh> P, const uint32_t* __restrict__ yp,
                  const uint32_t* __restrict__ yq, size_t count, uint32_t* __restrict__ out,
                  uint32_t* __restrict__ scratch, size_t ebase) {
  constexpr int Lp = Lh / 2;
  const Layout ly(1);
  const int SW = 2 * Lh + 4;
  const Col X = ly.slot(scratch, 0 * SW), A = ly.slot(scratch, 1 * SW), B = ly.slot(scratch, 2 * SW),
            C = ly.slot(scratch, 3 * SW), TT = ly.slot(scratch, 4 * SW), MP = ly.slot(scratch, 5 * SW),
            MQ = ly.slot(scratch, 6 * SW);
  for (size_t base = (size_t)blockIdx.x * ly.G; base < count; base += (size_t)ly.Gtot) {
    size_t e = base + ly.gl;
    const bool valid = e < count;
    if (!valid) e = count - 1;
    for (int h = 0; h < 2; ++h) {
      const ModConst<Lh>& M = h ? P.mq : P.mp;
      const uint32_t* y = h ? yq : yp;
      const Col& OUT = h ? MQ : MP;
      for (int j = 0; j < Lh; ++j) A[j] = y[tiled_index(e, j, Lh)];  // c^(h-1) R mod h^2
      g_zero(B, Lh);
      B[0] = 1u;
      g_mont(C, A, B, M.n, M.np, Lh, TT);  // x = c^(h-1) mod h^2, x = 1 mod h
      uint64_t br = 1;
      for (int j = 0; j < Lh && br; ++j) {
        const uint32_t v = C[j];
        C[j] = v - 1u;
        br = (v == 0u);
      }
      g_mul_lo(A, C, PArr{h ? P.qinvlo : P.pinvlo}, Lp);  // L_h(x) = (x-1)/h exactly
      g_copy_param(B, h ? P.hqR : P.hpR, Lp);
      g_mont(OUT, A, B, h ? P.q : P.p, h ? P.qnp : P.pnp, Lp, TT);  // m_h
    }
    // Garner: m = m_p + p [(m_q - m_p) p^-1 mod q]  (m_p < p < q)
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
    if (valid) write_tiled<1>(out, ebase + e, X, Lh, Grp<1>());
  }
}

// ------------------------------------------------------------------ launchers
namespace {

template <class K>
int grid_of(K kern, size_t smem, int sms) {
  int per = 0;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kThreads, smem) != cudaSuccess || per < 1) return -1;
  return per * sms;
}

// The power of all `count` elements of x (in place) by schedule E mod M.
int launch_power(const tc::Mod& M, const Sched<kMaxSchedHalf>& E, uint32_t* x, size_t count, uint32_t* tabs,
                 size_t tab_words, int* status, int sms, cudaStream_t st) {
  static thread_local TcExpParams P;
  P.m = M;
  P.e = E;
  if (cudaFuncSetAttribute(k_modexp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmem) != cudaSuccess)
    return PC2_ECUDA;
  const size_t tiles = (count + tc::kTileE - 1) / tc::kTileE;
  size_t grid = tiles < (size_t)(2 * sms) ? tiles : (size_t)(2 * sms);
  const size_t per_cta = (size_t)((1 << (E.w - 1)) + 1) * tc::kL * tc::kTileE;
  if (grid * per_cta > tab_words) return PC2_ENOMEM;
  k_modexp_tc<<<(unsigned)grid, tc::kThreads, tc::kSmem, st>>>(P, x, count, tabs, status);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

size_t power_scratch_words(int w, int sms) {
  return (size_t)2 * sms * ((size_t)(1 << (w - 1)) + 1) * tc::kL * tc::kTileE;
}

}  // namespace

int launch_enc_crt_tc(const EncCrtParams<64>& P, const TcKeyMods& K, const uint64_t* m64, const uint32_t* mwide,
                      size_t count, uint32_t* out, ScratchFn scratch_fn, void* sctx, int* status, int sms,
                      cudaStream_t st, size_t base, cudaEvent_t* ev) {
  constexpr int Lh = 64;
  const size_t smem = (size_t)Lh * kThreads * 4;
  auto pre = k_enc_tc_pre<Lh>;
  auto post = k_enc_tc_post<Lh>;
  const int gpre = grid_of(pre, smem, sms), gpost = grid_of(post, 0, sms);
  if (gpre < 0 || gpost < 0) return PC2_ECUDA;
  const int wpre = P.lp.e1.w > P.lq.e1.w ? P.lp.e1.w : P.lq.e1.w;
  const int tabw = (1 << (wpre - 1)) * Lh;
  const size_t pre_words = ((size_t)tabw + 5 * (size_t)(2 * Lh + 4)) * (size_t)gpre * kThreads;
  const size_t post_words = 8 * (size_t)(2 * Lh + 4) * (size_t)gpost * kThreads;
  const int wpow = P.lp.e2.w > P.lq.e2.w ? P.lp.e2.w : P.lq.e2.w;
  const size_t pow_words = power_scratch_words(wpow, sms);
  size_t work = pre_words > post_words ? pre_words : post_words;
  work = work > pow_words ? work : pow_words;
  const size_t vec = ((count + 31) / 32) * 32 * Lh;  // one tiled 64-word vector
  uint32_t* scratch = scratch_fn(sctx, (2 * vec + work) * 4);
  if (!scratch) return PC2_ENOMEM;
  uint32_t* sp = scratch;
  uint32_t* sq = scratch + vec;
  uint32_t* ws = scratch + 2 * vec;
  if (ev) cudaEventRecord(ev[0], st);
  pre<<<gpre, kThreads, smem, st>>>(P, count, sp, sq, ws, tabw);
  if (cudaGetLastError() != cudaSuccess) return PC2_ECUDA;
  if (ev) cudaEventRecord(ev[1], st);
  int rc = launch_power(K.p2, P.lp.e2, sp, count, ws, work, status, sms, st);
  if (ev) cudaEventRecord(ev[2], st);
  if (rc == PC2_OK) rc = launch_power(K.q2, P.lq.e2, sq, count, ws, work, status, sms, st);
  if (ev) cudaEventRecord(ev[3], st);
  if (rc != PC2_OK) return rc;
  post<<<gpost, kThreads, 0, st>>>(P, m64, mwide, count, sp, sq, out, ws, status, base);
  if (ev) cudaEventRecord(ev[4], st);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

int launch_dec_crt_tc(const DecParams<64>& P, const TcKeyMods& K, const uint32_t* ct, size_t count, uint32_t* out,
                      ScratchFn scratch_fn, void* sctx, int* status, int sms, cudaStream_t st, size_t base,
                      cudaEvent_t* ev) {
  constexpr int Lh = 64;
  auto pre = k_dec_tc_pre<Lh>;
  auto post = k_dec_tc_post<Lh>;
  const int gpre = grid_of(pre, 0, sms), gpost = grid_of(post, 0, sms);
  if (gpre < 0 || gpost < 0) return PC2_ECUDA;
  const size_t pre_words = 5 * (size_t)(2 * Lh + 4) * (size_t)gpre * kThreads;
  const size_t post_words = 7 * (size_t)(2 * Lh + 4) * (size_t)gpost * kThreads;
  const int wpow = P.ep.w > P.eq.w ? P.ep.w : P.eq.w;
  const size_t pow_words = power_scratch_words(wpow, sms);
  size_t work = pre_words > post_words ? pre_words : post_words;
  work = work > pow_words ? work : pow_words;
  const size_t vec = ((count + 31) / 32) * 32 * Lh;
  uint32_t* scratch = scratch_fn(sctx, (2 * vec + work) * 4);
  if (!scratch) return PC2_ENOMEM;
  uint32_t* sp = scratch;
  uint32_t* sq = scratch + vec;
  uint32_t* ws = scratch + 2 * vec;
  if (ev) cudaEventRecord(ev[0], st);
  pre<<<gpre, kThreads, 0, st>>>(P, ct, count, sp, sq, ws, base);
  if (cudaGetLastError() != cudaSuccess) return PC2_ECUDA;
  if (ev) cudaEventRecord(ev[1], st);
  int rc = launch_power(K.p2, P.ep, sp, count, ws, work, status, sms, st);
  if (ev) cudaEventRecord(ev[2], st);
  if (rc == PC2_OK) rc = launch_power(K.q2, P.eq, sq, count, ws, work, status, sms, st);
  if (ev) cudaEventRecord(ev[3], st);
  if (rc != PC2_OK) return rc;
  post<<<gpost, kThreads, 0, st>>>(P, sp, sq, count, out, ws, base);
  if (ev) cudaEventRecord(ev[4], st);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

// ------------------------------------------------------------------ host: the constant blocks
namespace tc {
namespace {

uint16_t bf16_of_digit(uint32_t d) {
  const float f = (float)d;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return (uint16_t)(u >> 16);  // exact: d < 256 needs 8 significant bits
}

// Slice of the Toeplitz matrix of a 256-digit operand: row n, K column kk
// holds digit n - kk when 0 <= n - kk < 256.
void toeplitz_slice(const uint32_t* w, int rows, uint16_t* out) {
  for (int n = 0; n < rows; ++n)
    for (int kk = 0; kk < 16; ++kk) {
      const int d = n - kk;
      const uint32_t v = (d >= 0 && d < 4 * kL) ? (w[d / 4] >> (8 * (d % 4))) & 0xffu : 0u;
      out[(kk / 8) * rows * 8 + n * 8 + (kk % 8)] = bf16_of_digit(v);
    }
}

// r = a b mod 2^(32 kL)
void mullo(const uint32_t* a, const uint32_t* b, uint32_t* r) {
  for (int j = 0; j < kL; ++j) r[j] = 0u;
  for (int i = 0; i < kL; ++i) {
    uint64_t c = 0;
    for (int j = 0; i + j < kL; ++j) {
      c += (uint64_t)a[i] * b[j] + r[i + j];
      r[i + j] = (uint32_t)c;
      c >>= 32;
    }
  }
}

}  // namespace

bool build_mod(const uint32_t* n64, Mod& M) {
  if (!(n64[0] & 1u)) return false;
  std::memcpy(M.n, n64, sizeof(M.n));
  // N^-1 mod 2^2048 by Newton's iteration x <- x (2 - N x), doubling the correct bits
  uint32_t inv[kL] = {}, t[kL], u[kL];
  uint32_t x0 = 1u;
  for (int i = 0; i < 5; ++i) x0 *= 2u - n64[0] * x0;  // mod 2^32
  inv[0] = x0;
  for (int it = 0; it < 6; ++it) {  // 32 -> 2048 correct bits
    mullo(inv, n64, t);
    uint64_t br = 0;  // u = 2 - t mod 2^2048
    for (int j = 0; j < kL; ++j) {
      const uint64_t s = j == 0 ? 2ull : 0ull, v = (uint64_t)t[j] + br;
      u[j] = (uint32_t)(s - v);
      br = s < v;
    }
    mullo(inv, u, t);
    std::memcpy(inv, t, sizeof(inv));
  }
  uint32_t np[kL];  // N' = 2^2048 - N^-1
  uint64_t br = 0;
  for (int j = 0; j < kL; ++j) {
    const uint64_t v = (uint64_t)inv[j] + br;
    np[j] = (uint32_t)(0ull - v);
    br = v != 0;
  }
  M.np0 = np[0];
  toeplitz_slice(np, kB1Rows, M.b1);
  toeplitz_slice(n64, kB2Rows, M.b2);
  return true;
}

}  // namespace tc
}  // namespace pc2
