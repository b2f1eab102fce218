// tc_paillier.cu -- key-owner encryption and CRT decryption at 2048-bit n
// with the full-width powers on the tensor-core Montgomery product
// (tc_core.cuh).
//
// Each operation runs as set-up, powers and finish:
//   pre   the per-element set-up of both CRT halves: for encryption r R_h
//         mod h (integer pipe), the lifted route's half-width power
//         s = r^(h' mod (h-1)) mod h (tensor cores, 32 limbs) and the lift
//         s R mod h^2 (integer pipe); for decryption c R mod h^2;
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
template <int L>
struct TcExpParams {
  tc::Mod<L> m;
  Sched<kMaxSchedHalf> e;
};
static_assert(sizeof(TcExpParams<64>) + 256 <= 32764, "parameter block too large");

// Resident CTAs per SM of the power kernel: two at 64 limbs (registers and
// the 64 KB A tile), four at 32 limbs (4 x 128 TMEM columns, 128 registers).
template <int L>
constexpr int tc_ctas() { return L == 64 ? 2 : 4; }

// x <- x^E (Montgomery domain, L words, tiled, in place).  tabs: per CTA
// (2^(w-1) + 1) entries of L words x 128 elements (odd powers, then x^2).
template <int L>
__global__ void __launch_bounds__(tc::kThreads, tc_ctas<L>())
    k_modexp_tc(const __grid_constant__ TcExpParams<L> P, uint32_t* __restrict__ xy, size_t count,
                uint32_t* __restrict__ tabs, int* status) {
  using Core = tc::Core<L>;
  extern __shared__ __align__(1024) uint8_t smem[];
  const tc::Smem s = Core::smem_layout(smem);
  const uint32_t tmem = Core::setup(s, P.m);
  {
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
        {
          // one reduction site for both product forms (a smaller loop body)
          uint32_t t[L];
          tc::Prod pr;
          if (src < 0) {
            pr = Core::product_sqr(a, t, s);
          } else {
            Core::write_b_global(s, entry(src), ts);
            pr = Core::product_rows(a, t, s);
          }
          Core::reduce(a, t, pr, s, tmem, P.m.n, st);
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
    if (!st.ok && status) atomicOr(status, PC2_ST_TIMEOUT);
  }
  Core::teardown(tmem);
}

// ------------------------------------------------------------------ encryption: set-up and finish
// a = (a + b) mod N for a, b < N (L words; a in registers, b a column).
template <int L>
__device__ __forceinline__ void add_mod_reg(uint32_t (&a)[L], const Col& b, const uint32_t* N) {
  uint64_t c = 0;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    c += (uint64_t)a[j] + b[j];
    a[j] = (uint32_t)c;
    c >>= 32;
  }
  uint32_t d[L];
  uint64_t br = 0;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const uint64_t t = (uint64_t)a[j] - N[j] - br;
    d[j] = (uint32_t)t;
    br = t >> 63;
  }
  const bool sub = c != 0 || br == 0;  // the sum is >= N
#pragma unroll
  for (int j = 0; j < L; ++j) a[j] = sub ? d[j] : a[j];
}

// Set-up 1: r R_h mod h for h = p, q (half width) from the raw draw X, the
// start of the lifted route of LiftConst.
template <int Lh>
__global__ void __launch_bounds__(kThreads, min_blocks(Lh, 1))
    k_enc_tc_pre1(const __grid_constant__ EncCrtParams<Lh> P, size_t count, uint32_t* __restrict__ rp,
                  uint32_t* __restrict__ rq, uint32_t* __restrict__ scratch) {
  constexpr int Lp = Lh / 2;
  extern __shared__ uint32_t pre_sh[];  // word i of this thread's operand at pre_sh[i * kThreads + tid]
  const Layout ly(1);
  const int SW = 2 * Lh + 4;
  const Col X = ly.slot(scratch, 0 * SW);
  const Grp<1> g;
  const Col bsh{pre_sh + threadIdx.x, kThreads};
  for (size_t base = (size_t)blockIdx.x * ly.G; base < count; base += (size_t)ly.Gtot) {
    size_t e = base + ly.gl;
    const bool valid = e < count;
    if (!valid) e = count - 1;
    const uint32_t sid = P.round_ptr ? ((*P.round_ptr << 8) | P.kind) : P.stream;
    gen_r(X, P.seed, sid, P.e0 + e, Lh + 2, 2 * Lh);
    for (int h = 0; h < 2; ++h) {
      const ModConst<Lp>& Hm = (h ? P.lq : P.lp).h;
      // r = x0 + x1 R_h (x0 = words 0..Lp-1, x1 = words Lp..2Lp+1 of the draw):
      // r R_h = x0 R_h + (x1 R_h) R_h mod h, Montgomery products in registers
      uint32_t a[Lp];
#pragma unroll
      for (int j = 0; j < Lp; ++j) a[j] = X[2 * Lp + j];  // x1's high words
      mont_mul<Lp, 1>(a, Hm.r3, 1, ParamN{Hm.n}, Hm.np, g);
#pragma unroll
      for (int j = 0; j < Lp; ++j) bsh[j] = a[j];
#pragma unroll
      for (int j = 0; j < Lp; ++j) a[j] = X[Lp + j];      // x1's low words
      mont_mul<Lp, 1>(a, Hm.r2, 1, ParamN{Hm.n}, Hm.np, g);
      add_mod_reg<Lp>(a, bsh, Hm.n);                      // x1 R_h mod h
      mont_mul<Lp, 1>(a, Hm.r2, 1, ParamN{Hm.n}, Hm.np, g);  // x1 R_h^2
#pragma unroll
      for (int j = 0; j < Lp; ++j) bsh[j] = a[j];
#pragma unroll
      for (int j = 0; j < Lp; ++j) a[j] = X[j];
      mont_mul<Lp, 1>(a, Hm.r2, 1, ParamN{Hm.n}, Hm.np, g);  // x0 R_h
      add_mod_reg<Lp>(a, bsh, Hm.n);                      // r R_h mod h
      uint32_t* out = h ? rq : rp;
      if (valid) {
#pragma unroll
        for (int j = 0; j < Lp; ++j) out[tiled_index(e, j, Lp)] = a[j];
      }
    }
  }
}

// Set-up 2: s R mod h^2 from s R_h (the half-width power's result), the lift
// of LiftConst: a Montgomery product with R_h^3 mod h^2.
template <int Lh>
__global__ void __launch_bounds__(kThreads, min_blocks(Lh, 1))
    k_enc_tc_pre2(const __grid_constant__ EncCrtParams<Lh> P, size_t count, const uint32_t* __restrict__ sp1,
                  const uint32_t* __restrict__ sq1, uint32_t* __restrict__ sp, uint32_t* __restrict__ sq,
                  uint32_t* __restrict__ scratch) {
  constexpr int Lp = Lh / 2;
  const Layout ly(1);
  const Grp<1> g;
  for (size_t base = (size_t)blockIdx.x * ly.G; base < count; base += (size_t)ly.Gtot) {
    size_t e = base + ly.gl;
    const bool valid = e < count;
    if (!valid) e = count - 1;
    for (int h = 0; h < 2; ++h) {
      const ModConst<Lh>& M = h ? P.mq : P.mp;
      const LiftConst<Lh>& H = h ? P.lq : P.lp;
      const uint32_t* in = h ? sq1 : sp1;
      uint32_t a[Lh];
#pragma unroll
      for (int j = 0; j < Lh; ++j) a[j] = j < Lp ? in[tiled_index(e, j, Lp)] : 0u;
      mont_mul<Lh, 1>(a, H.lift, 1, ParamN{M.n}, M.np, g);  // s R mod h^2
      uint32_t* out = h ? sq : sp;
      if (valid) {
#pragma unroll
        for (int j = 0; j < Lh; ++j) out[tiled_index(e, j, Lh)] = a[j];
      }
    }
  }
}

// Finish: c = (1 + m n) (r^n mod h^2) mod h^2 per half, then Eq. (gA-C-B).
// The Montgomery products run in registers (the library's CIOS product, the
// second operand in a shared-memory column of this thread or in the
// parameter block); 1 + m n and the recombination's full product use the
// word-serial glue columns.
template <int Lh>
__global__ void __launch_bounds__(kThreads, min_blocks(Lh, 1))
    k_enc_tc_post(const __grid_constant__ EncCrtParams<Lh> P, const uint64_t* __restrict__ m64,
                  const uint32_t* __restrict__ mwide, size_t count, const uint32_t* __restrict__ yp,
                  const uint32_t* __restrict__ yq, uint32_t* __restrict__ out, uint32_t* __restrict__ scratch,
                  int* status, size_t base_out) {
  extern __shared__ uint32_t post_sh[];  // word i of this thread's operand at post_sh[i * kThreads + tid]
  const Layout ly(1);
  const int SW = 2 * Lh + 4;
  const Col X = ly.slot(scratch, 0 * SW), GM = ly.slot(scratch, 1 * SW), A = ly.slot(scratch, 2 * SW),
            C = ly.slot(scratch, 4 * SW), CP = ly.slot(scratch, 6 * SW), CQ = ly.slot(scratch, 7 * SW);
  const Grp<1> g;
  const Col bsh{post_sh + threadIdx.x, kThreads};
  for (size_t base = (size_t)blockIdx.x * ly.G; base < count; base += (size_t)ly.Gtot) {
    size_t e = base + ly.gl;
    const bool valid = e < count;
    if (!valid) e = count - 1;
    make_gm(GM, A, m64, mwide, e, P.nwords, Lh, 2 * Lh, valid, status);  // 1 + m n, 2 Lh words
    for (int h = 0; h < 2; ++h) {
      const ModConst<Lh>& M = h ? P.mq : P.mp;
      const uint32_t* y = h ? yq : yp;
      const Col& OUT = h ? CQ : CP;
      uint32_t a[Lh];
      // (1 + m n) R mod h^2 = mont(lo, R^2) + mont(hi, R^3)
#pragma unroll
      for (int j = 0; j < Lh; ++j) a[j] = GM[Lh + j];
      mont_mul<Lh, 1>(a, M.r3, 1, ParamN{M.n}, M.np, g);
#pragma unroll
      for (int j = 0; j < Lh; ++j) bsh[j] = a[j];
#pragma unroll
      for (int j = 0; j < Lh; ++j) a[j] = GM[j];
      mont_mul<Lh, 1>(a, M.r2, 1, ParamN{M.n}, M.np, g);
      add_mod_reg<Lh>(a, bsh, M.n);
#pragma unroll
      for (int j = 0; j < Lh; ++j) bsh[j] = a[j];                   // (1 + m n) R mod h^2
#pragma unroll
      for (int j = 0; j < Lh; ++j) a[j] = y[tiled_index(e, j, Lh)];  // (r^n mod h^2) R
      mont_mul<Lh, 1>(a, bsh.p, bsh.s, ParamN{M.n}, M.np, g);       // c_h R
#pragma unroll
      for (int j = 0; j < Lh; ++j) bsh[j] = j == 0 ? 1u : 0u;
      mont_mul<Lh, 1>(a, bsh.p, bsh.s, ParamN{M.n}, M.np, g);       // c_h
#pragma unroll
      for (int j = 0; j < Lh; ++j) OUT[j] = a[j];
    }
    // Eq. (gA-C-B): c = c_p + [(c_q - c_p) (p^2)^-1 mod q^2] p^2  (c_p < p^2 < q^2)
    if (g_sub(A, CQ, CP, Lh)) g_add(A, A, PArr{P.mq.n}, Lh);
    {
      uint32_t a[Lh];
#pragma unroll
      for (int j = 0; j < Lh; ++j) a[j] = A[j];
      mont_mul<Lh, 1>(a, P.pinv2R, 1, ParamN{P.mq.n}, P.mq.np, g);
#pragma unroll
      for (int j = 0; j < Lh; ++j) C[j] = a[j];
    }
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
  extern __shared__ uint32_t dpre_sh[];  // word i of this thread's operand at dpre_sh[i * kThreads + tid]
  const Layout ly(1);
  const Grp<1> g;
  const Col bsh{dpre_sh + threadIdx.x, kThreads};
  for (size_t base = (size_t)blockIdx.x * ly.G; base < count; base += (size_t)ly.Gtot) {
    size_t e = base + ly.gl;
    const bool valid = e < count;
    if (!valid) e = count - 1;
    for (int h = 0; h < 2; ++h) {
      const ModConst<Lh>& M = h ? P.mq : P.mp;
      // c R mod h^2 = mont(c_lo, R^2) + mont(c_hi, R^3), products in registers
      uint32_t a[Lh];
#pragma unroll
      for (int j = 0; j < Lh; ++j) a[j] = ct[tiled_index(ebase + e, Lh + j, 2 * Lh)];
      mont_mul<Lh, 1>(a, M.r3, 1, ParamN{M.n}, M.np, g);
#pragma unroll
      for (int j = 0; j < Lh; ++j) bsh[j] = a[j];
#pragma unroll
      for (int j = 0; j < Lh; ++j) a[j] = ct[tiled_index(ebase + e, j, 2 * Lh)];
      mont_mul<Lh, 1>(a, M.r2, 1, ParamN{M.n}, M.np, g);
      add_mod_reg<Lh>(a, bsh, M.n);
      uint32_t* s = h ? sq : sp;
      if (valid) {
#pragma unroll
        for (int j = 0; j < Lh; ++j) s[tiled_index(e, j, Lh)] = a[j];
      }
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
template <int L>
int launch_power(const tc::Mod<L>& M, const Sched<kMaxSchedHalf>& E, uint32_t* x, size_t count, uint32_t* tabs,
                 size_t tab_words, int* status, int sms, cudaStream_t st) {
  static thread_local TcExpParams<L> P;
  P.m = M;
  P.e = E;
  auto kern = k_modexp_tc<L>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::Core<L>::kSmem) != cudaSuccess)
    return PC2_ECUDA;
  const size_t tiles = (count + tc::kTileE - 1) / tc::kTileE;
  const size_t cap = (size_t)tc_ctas<L>() * sms;
  const size_t grid = tiles < cap ? tiles : cap;
  const size_t per_cta = (size_t)((1 << (E.w - 1)) + 1) * L * tc::kTileE;
  if (grid * per_cta > tab_words) return PC2_ENOMEM;
  kern<<<(unsigned)grid, tc::kThreads, tc::Core<L>::kSmem, st>>>(P, x, count, tabs, status);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

template <int L>
size_t power_scratch_words(int w, int sms) {
  return (size_t)tc_ctas<L>() * sms * ((size_t)(1 << (w - 1)) + 1) * L * tc::kTileE;
}

}  // namespace

int launch_enc_crt_tc(const EncCrtParams<64>& P, const TcKeyMods& K, const uint64_t* m64, const uint32_t* mwide,
                      size_t count, uint32_t* out, ScratchFn scratch_fn, void* sctx, int* status, int sms,
                      cudaStream_t st, size_t base, cudaEvent_t* ev) {
  constexpr int Lh = 64, Lp = 32;
  auto pre1 = k_enc_tc_pre1<Lh>;
  auto pre2 = k_enc_tc_pre2<Lh>;
  auto post = k_enc_tc_post<Lh>;
  const size_t post_smem = (size_t)Lh * kThreads * 4;  // one operand column per thread
  const size_t pre1_smem = (size_t)Lp * kThreads * 4;
  const int g1 = grid_of(pre1, pre1_smem, sms), g2 = grid_of(pre2, 0, sms), gpost = grid_of(post, post_smem, sms);
  if (g1 < 0 || g2 < 0 || gpost < 0) return PC2_ECUDA;
  const size_t sw = 2 * Lh + 4;
  const size_t glue = 8 * sw * (size_t)(g1 > gpost ? (g1 > g2 ? g1 : g2) : (gpost > g2 ? gpost : g2)) * kThreads;
  const int w1 = P.lp.e1.w > P.lq.e1.w ? P.lp.e1.w : P.lq.e1.w;
  const int w2 = P.lp.e2.w > P.lq.e2.w ? P.lp.e2.w : P.lq.e2.w;
  const size_t pw1 = power_scratch_words<Lp>(w1, sms), pw2 = power_scratch_words<Lh>(w2, sms);
  size_t work = glue > pw1 ? glue : pw1;
  work = work > pw2 ? work : pw2;
  const size_t tiles = (count + 31) / 32 * 32;
  const size_t vec = tiles * Lh, vec1 = tiles * Lp;  // tiled vectors of 64 and 32 words
  uint32_t* scratch = scratch_fn(sctx, (2 * vec + 2 * vec1 + work) * 4);
  if (!scratch) return PC2_ENOMEM;
  uint32_t* sp = scratch;
  uint32_t* sq = sp + vec;
  uint32_t* sp1 = sq + vec;
  uint32_t* sq1 = sp1 + vec1;
  uint32_t* ws = sq1 + vec1;
  if (ev) cudaEventRecord(ev[0], st);
  pre1<<<g1, kThreads, pre1_smem, st>>>(P, count, sp1, sq1, ws);
  if (cudaGetLastError() != cudaSuccess) return PC2_ECUDA;
  int rc = launch_power<Lp>(K.p, P.lp.e1, sp1, count, ws, work, status, sms, st);  // s R_h mod p
  if (rc == PC2_OK) rc = launch_power<Lp>(K.q, P.lq.e1, sq1, count, ws, work, status, sms, st);
  if (rc != PC2_OK) return rc;
  pre2<<<g2, kThreads, 0, st>>>(P, count, sp1, sq1, sp, sq, ws);
  if (cudaGetLastError() != cudaSuccess) return PC2_ECUDA;
  if (ev) cudaEventRecord(ev[1], st);
  rc = launch_power<Lh>(K.p2, P.lp.e2, sp, count, ws, work, status, sms, st);  // (r^n mod p^2) R
  if (ev) cudaEventRecord(ev[2], st);
  if (rc == PC2_OK) rc = launch_power<Lh>(K.q2, P.lq.e2, sq, count, ws, work, status, sms, st);
  if (ev) cudaEventRecord(ev[3], st);
  if (rc != PC2_OK) return rc;
  post<<<gpost, kThreads, post_smem, st>>>(P, m64, mwide, count, sp, sq, out, ws, status, base);
  if (ev) cudaEventRecord(ev[4], st);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

int launch_dec_crt_tc(const DecParams<64>& P, const TcKeyMods& K, const uint32_t* ct, size_t count, uint32_t* out,
                      ScratchFn scratch_fn, void* sctx, int* status, int sms, cudaStream_t st, size_t base,
                      cudaEvent_t* ev) {
  constexpr int Lh = 64;
  auto pre = k_dec_tc_pre<Lh>;
  auto post = k_dec_tc_post<Lh>;
  const size_t dpre_smem = (size_t)Lh * kThreads * 4;  // one operand column per thread
  const int gpre = grid_of(pre, dpre_smem, sms), gpost = grid_of(post, 0, sms);
  if (gpre < 0 || gpost < 0) return PC2_ECUDA;
  const size_t pre_words = 5 * (size_t)(2 * Lh + 4) * (size_t)gpre * kThreads;
  const size_t post_words = 7 * (size_t)(2 * Lh + 4) * (size_t)gpost * kThreads;
  const int wpow = P.ep.w > P.eq.w ? P.ep.w : P.eq.w;
  const size_t pow_words = power_scratch_words<Lh>(wpow, sms);
  size_t work = pre_words > post_words ? pre_words : post_words;
  work = work > pow_words ? work : pow_words;
  const size_t vec = ((count + 31) / 32) * 32 * Lh;
  uint32_t* scratch = scratch_fn(sctx, (2 * vec + work) * 4);
  if (!scratch) return PC2_ENOMEM;
  uint32_t* sp = scratch;
  uint32_t* sq = scratch + vec;
  uint32_t* ws = scratch + 2 * vec;
  if (ev) cudaEventRecord(ev[0], st);
  pre<<<gpre, kThreads, dpre_smem, st>>>(P, ct, count, sp, sq, ws, base);
  if (cudaGetLastError() != cudaSuccess) return PC2_ECUDA;
  if (ev) cudaEventRecord(ev[1], st);
  int rc = launch_power<Lh>(K.p2, P.ep, sp, count, ws, work, status, sms, st);
  if (ev) cudaEventRecord(ev[2], st);
  if (rc == PC2_OK) rc = launch_power<Lh>(K.q2, P.eq, sq, count, ws, work, status, sms, st);
  if (ev) cudaEventRecord(ev[3], st);
  if (rc != PC2_OK) return rc;
  post<<<gpost, kThreads, 0, st>>>(P, sp, sq, count, out, ws, base);
  if (ev) cudaEventRecord(ev[4], st);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

// ------------------------------------------------------------------ host: the constant blocks
namespace tc {
namespace {

// The f16 bits of a digit 0..255 (exact: at most 8 significant bits).
uint16_t f16_of_digit(uint32_t d) {
  if (d == 0) return 0;
  const int e = 31 - __builtin_clz(d);  // d = 2^e (1 + f), f < 1
  return (uint16_t)(((e + 15) << 10) | ((d << (10 - e)) & 0x3ffu));
}

// Slice of the Toeplitz matrix of a 4L-digit operand w: row n, K column kk
// holds digit n - kk when 0 <= n - kk < 4L.
template <int L>
void toeplitz_slice(const uint32_t* w, int rows, uint16_t* out) {
  for (int n = 0; n < rows; ++n)
    for (int kk = 0; kk < 16; ++kk) {
      const int d = n - kk;
      const uint32_t v = (d >= 0 && d < 4 * L) ? (w[d / 4] >> (8 * (d % 4))) & 0xffu : 0u;
      out[(kk / 8) * rows * 8 + n * 8 + (kk % 8)] = f16_of_digit(v);
    }
}

// r = a b mod 2^(32 L)
template <int L>
void mullo(const uint32_t* a, const uint32_t* b, uint32_t* r) {
  for (int j = 0; j < L; ++j) r[j] = 0u;
  for (int i = 0; i < L; ++i) {
    uint64_t c = 0;
    for (int j = 0; i + j < L; ++j) {
      c += (uint64_t)a[i] * b[j] + r[i + j];
      r[i + j] = (uint32_t)c;
      c >>= 32;
    }
  }
}

}  // namespace

template <int L>
bool build_mod(const uint32_t* n, Mod<L>& M) {
  if (!(n[0] & 1u)) return false;
  std::memcpy(M.n, n, sizeof(M.n));
  // N^-1 mod 2^(32 L) by Newton's iteration x <- x (2 - N x), doubling the correct bits
  uint32_t inv[L] = {}, t[L], u[L];
  uint32_t x0 = 1u;
  for (int i = 0; i < 5; ++i) x0 *= 2u - n[0] * x0;  // mod 2^32
  inv[0] = x0;
  for (int it = 0; it < 6; ++it) {  // 32 -> 2048 correct bits
    mullo<L>(inv, n, t);
    uint64_t br = 0;  // u = 2 - t mod 2^(32 L)
    for (int j = 0; j < L; ++j) {
      const uint64_t s2 = j == 0 ? 2ull : 0ull, v = (uint64_t)t[j] + br;
      u[j] = (uint32_t)(s2 - v);
      br = s2 < v;
    }
    mullo<L>(inv, u, t);
    std::memcpy(inv, t, sizeof(inv));
  }
  uint32_t np[L];  // N' = 2^(32 L) - N^-1
  uint64_t br = 0;
  for (int j = 0; j < L; ++j) {
    const uint64_t v = (uint64_t)inv[j] + br;
    np[j] = (uint32_t)(0ull - v);
    br = v != 0;
  }
  M.np0 = np[0];
  toeplitz_slice<L>(np, 4 * L, M.b1);
  toeplitz_slice<L>(n, 4 * L + 16, M.b2);
  return true;
}
template bool build_mod<32>(const uint32_t*, Mod<32>&);
template bool build_mod<64>(const uint32_t*, Mod<64>&);

}  // namespace tc
}  // namespace pc2
