// paillier_kernels.cuh -- the Paillier kernels of libpc2 and their launchers.
//
//   k_enc_crt  key-owner encryption, Eq. (itq1) evaluated through the CRT
//              split of Sec. IV-A: r^n mod p^2 and mod q^2 (by the lifted
//              route of LiftConst, or with the exponent reduced mod phi(p^2),
//              phi(q^2) as in Lemma 1 when a lane would hold fewer than two
//              half-width limbs), each half times g^m = 1 + m n, recombined
//              by Eq. (gA-C-B) (Lemma 2).
//   k_enc_pub  public-key encryption, Eq. (itq1) directly mod n^2.
//   k_dec_crt  decryption of Sec. III-C via the CRT: m_p = L_p(c^(p-1) mod p^2) h_p
//              mod p, m_q likewise, Garner recombination mod n (equal to
//              L(c^lambda mod n^2) mu mod n; Sec. IV-A notes the same CRT
//              acceleration applies to c^lambda).
//   k_hom_sum  Definition 1 over several operands: prod_g c_g mod n^2.
//   k_hom_scal Definition 2: c^k mod n^2, per-element k < 2^64.
//   k_hom_scal_wide  Definition 2 with a full-width scalar k < 2^nbits.
//
// All modexp kernels are persistent: a grid of (SMs x resident CTAs) walks the
// elements; each element is owned by a group of T lanes (mont.cuh).  Scratch
// (global memory, from the context) holds each group's window table and glue
// columns, interleaved by group so that a warp's accesses coalesce.
#pragma once
#include <cuda_runtime.h>

#include "mont.cuh"
#include "pc2_kernels.h"
#include "philox.h"

namespace pc2 {

// ------------------------------------------------------------------ helpers
template <int S, int T, int MAXS>
__device__ __forceinline__ void run_modexp(uint32_t (&a)[S], const Sched<MAXS>& E, const uint32_t* n, uint32_t np,
                                           const Col& tab, const Col& bsh, const Grp<T>& g) {
  if constexpr (T == 1) {
    modexp_sched<S, T>(a, E, tab, bsh, ParamN{n}, np, g);
  } else {
    const RegN<S> rn = reg_n<S, T>(n, g);
    modexp_sched<S, T>(a, E, tab, bsh, rn, np, g);
  }
}

// r_raw for element e: `words` Philox words, zero-padded to `total`.
__device__ __forceinline__ void gen_r(const Col& X, uint64_t seed, uint32_t stream, uint64_t e, int words, int total) {
  for (int j4 = 0; 4 * j4 < words; ++j4) {
    const U4 v = r_block(seed, stream, e, (uint32_t)j4);
    const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (4 * j4 + i < words) X[4 * j4 + i] = w4[i];
  }
  for (int j = words; j < total; ++j) X[j] = 0u;
}

// GM = 1 + m n (zero-padded to `total` words); m from uint64 input or a tiled
// wide input of Ln limbs.  Flags PC2_ST_RANGE when a wide m >= n.
__device__ __forceinline__ void make_gm(const Col& GM, const Col& M, const uint64_t* m64, const uint32_t* mwide,
                                        size_t e, const uint32_t* n, int Ln, int total, bool valid, int* status) {
  int mw;
  if (mwide) {
    for (int j = 0; j < Ln; ++j) M[j] = mwide[tiled_index(e, j, Ln)];
    mw = Ln;
    if (valid && g_ge(M, PArr{n}, Ln)) atomicOr(status, PC2_ST_RANGE);
  } else {
    const uint64_t m = m64[e];
    M[0] = (uint32_t)m;
    M[1] = (uint32_t)(m >> 32);
    mw = 2;
  }
  g_mul(GM, M, mw, PArr{n}, Ln);
  uint64_t c = 1;
  for (int j = 0; j < mw + Ln; ++j) {
    c += GM[j];
    GM[j] = (uint32_t)c;
    c >>= 32;
  }
  for (int j = mw + Ln; j < total; ++j) GM[j] = 0u;
}

// Writes words [0, Lc) of column V as element e of a tiled output; lane k of
// the group writes its share of the words.
template <int T>
__device__ __forceinline__ void write_tiled(uint32_t* out, size_t e, const Col& V, int Lc, const Grp<T>& g) {
  const int per = Lc / T;
  for (int j = g.k * per; j < (g.k + 1) * per; ++j) out[tiled_index(e, j, Lc)] = V[j];
}

struct Layout {
  int G, gl, Gtot, gg;
  __device__ Layout(int T) {
    G = (int)blockDim.x / T;
    gl = (int)threadIdx.x / T;
    Gtot = (int)gridDim.x * G;
    gg = (int)blockIdx.x * G + gl;
  }
  __device__ __forceinline__ Col slot(uint32_t* scratch, size_t first_word) const {
    return Col{scratch + first_word * (size_t)Gtot + gg, Gtot};
  }
};

// ------------------------------------------------------------------ CRT encryption
// A = (r^n mod h^2) R by the lifted route (LiftConst): r mod h from the raw
// draw X (words [0, Lh + 2)), s = r^(h' mod (h-1)) mod h at half width, then
// s^h mod h^2.  Uses columns A, B, C, TT; X is read only.  nfast, hfast: h^2
// and h where one-lane products read them (compile-time offsets into the
// parameter block or constant memory); with T > 1 each lane loads its
// segment of M.n, H.h.n into registers.
template <int Lh, int T>
__device__ __forceinline__ void rn_lifted(const ModConst<Lh>& M, const uint32_t* nfast, const LiftConst<Lh>& H,
                                          const uint32_t* hfast, const Col& X, const Col& A, const Col& B,
                                          const Col& C, const Col& TT, const Col& tab, const Col& bsh,
                                          const Grp<T>& g) {
  constexpr int Lp = Lh / 2, Sa = Lp / T, S = Lh / T;
  // r = x0 + x1 R_h with x0 = words [0, Lp), x1 = words [Lp, 3 Lp) < R_h^2:
  // r R_h = x0 R_h + (x1 R_h) R_h mod h
  grp_to_mont_2l<Lp, T>(A, X.off(Lp), H.h.n, H.h.r2, H.h.r3, H.h.np, B, C, TT, g);  // x1 R_h
  grp_mont<Lp, T>(A, A, const_col(H.h.r2), H.h.n, H.h.np, TT, g);                  // x1 R_h^2
  grp_mont<Lp, T>(C, X, const_col(H.h.r2), H.h.n, H.h.np, TT, g);                  // x0 R_h
  g_addmod(A, A, C, H.h.n, Lp);                                                    // r R_h mod h
  __syncwarp();
  {
    uint32_t a[Sa];
    load_seg(a, A, g);
    run_modexp<Sa, T>(a, H.e1, T == 1 ? hfast : H.h.n, H.h.np, tab, bsh, g);  // s R_h
    store_seg(A, a, g);
  }
  __syncwarp();
  for (int j = Lp; j < Lh; ++j) A[j] = 0u;
  grp_mont<Lh, T>(A, A, const_col(H.lift), M.n, M.np, TT, g);             // s R mod h^2
  __syncwarp();
  uint32_t a[S];
  load_seg(a, A, g);
  run_modexp<S, T>(a, H.e2, T == 1 ? nfast : M.n, M.np, tab, bsh, g);      // s^h R = (r^n mod h^2) R
  store_seg(A, a, g);
  __syncwarp();
}

template <int Lh, int T>
__device__ __forceinline__ void enc_half(const ModConst<Lh>& M, const Sched<kMaxSched>& E, const LiftConst<Lh>& H,
                                         const Col& X, const Col& GM, const Col& OUT, const Col& A, const Col& B,
                                         const Col& C, const Col& TT, const Col& tab, const Col& bsh,
                                         const Grp<T>& g) {
  constexpr int S = Lh / T;
  if constexpr (lift_route<Lh, T>()) {
    rn_lifted<Lh, T>(M, M.n, H, H.h.n, X, A, B, C, TT, tab, bsh, g);
  } else {
    // direct route: the power by n mod h(h-1)
    grp_to_mont_2l<Lh, T>(A, X, M.n, M.r2, M.r3, M.np, B, C, TT, g);  // r~ = r R mod h^2
    __syncwarp();
    uint32_t a[S];
    load_seg(a, A, g);
    run_modexp<S, T>(a, E, M.n, M.np, tab, bsh, g);          // (r^n mod h^2) R
    store_seg(A, a, g);
    __syncwarp();
  }
  grp_to_mont_2l<Lh, T>(B, GM, M.n, M.r2, M.r3, M.np, C, OUT, TT, g);  // (1 + m n) R mod h^2
  grp_mont<Lh, T>(C, A, B, M.n, M.np, TT, g);                          // c_h R
  g_zero(B, Lh);
  B[0] = 1u;
  grp_mont<Lh, T>(OUT, C, B, M.n, M.np, TT, g);                        // c_h
}

template <int Lh, int T>
__global__ void __launch_bounds__(kThreads, min_blocks(Lh, T)) k_enc_crt(const __grid_constant__ EncCrtParams<Lh> P,
                                                      const uint64_t* __restrict__ m64,
                                                      const uint32_t* __restrict__ mwide, size_t count,
                                                      uint32_t* __restrict__ out, uint32_t* __restrict__ scratch,
                                                      int tabw, int* status, size_t base_out) {
  extern __shared__ uint32_t bsh_all[];
  const Grp<T> g;
  const Layout ly(T);
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
    const uint32_t sid = P.round_ptr ? ((*P.round_ptr << 8) | P.kind) : P.stream;
    gen_r(X, P.seed, sid, P.e0 + e, Lh + 2, 2 * Lh);
    make_gm(GM, A, m64, mwide, e, P.nwords, Lh, 2 * Lh, valid, status);
    enc_half<Lh, T>(P.mp, P.ep, P.lp, X, GM, CP, A, B, C, TT, tab, bsh, g);
    enc_half<Lh, T>(P.mq, P.eq, P.lq, X, GM, CQ, A, B, C, TT, tab, bsh, g);
    // Eq. (gA-C-B): c = c_p + [(c_q - c_p) (p^2)^-1 mod q^2] p^2  (c_p < p^2 < q^2)
    if (g_sub(A, CQ, CP, Lh)) g_add(A, A, PArr{P.mq.n}, Lh);
    grp_mont<Lh, T>(C, A, const_col(P.pinv2R), P.mq.n, P.mq.np, TT, g);
    g_mul(X, C, Lh, PArr{P.p2}, Lh);
    uint64_t c = 0;
    for (int j = 0; j < 2 * Lh; ++j) {
      c += (uint64_t)X[j] + (j < Lh ? CP[j] : 0u);
      X[j] = (uint32_t)c;
      c >>= 32;
    }
    if (valid) write_tiled<T>(out, base_out + e, X, 2 * Lh, g);
    __syncwarp();
  }
}

// ------------------------------------------------------------------ public-key encryption
template <int L2, int T>
__global__ void __launch_bounds__(kThreads, min_blocks(L2, T)) k_enc_pub(const __grid_constant__ EncPubParams<L2> P,
                                                      const uint64_t* __restrict__ m64,
                                                      const uint32_t* __restrict__ mwide, size_t count,
                                                      uint32_t* __restrict__ out, uint32_t* __restrict__ scratch,
                                                      int tabw, int* status) {
  constexpr int S = L2 / T, Ln = L2 / 2;
  extern __shared__ uint32_t bsh_all[];
  const Grp<T> g;
  const Layout ly(T);
  const Col bsh{bsh_all + ly.gl, ly.G};
  const Col tab = ly.slot(scratch, 0);
  const int SW = L2 + 4;
  const Col X = ly.slot(scratch, tabw + 0 * SW), GM = ly.slot(scratch, tabw + 1 * SW),
            A = ly.slot(scratch, tabw + 2 * SW), TT = ly.slot(scratch, tabw + 3 * SW);
  for (size_t base = (size_t)blockIdx.x * ly.G; base < count; base += (size_t)ly.Gtot) {
    size_t e = base + ly.gl;
    const bool valid = e < count;
    if (!valid) e = count - 1;
    gen_r(X, P.seed, P.stream, P.e0 + e, Ln + 2, L2);
    __syncwarp();
    uint32_t a[S];
    load_seg(a, X, g);
    // r~ = r R mod n^2  (r_raw < R)
#pragma unroll
    for (int j = 0; j < S; ++j) bsh[g.k * S + j] = P.m.r2[g.k * S + j];
    __syncwarp();
    if constexpr (T == 1) {
      mont_mul<S, T>(a, bsh.p, bsh.s, ParamN{P.m.n}, P.m.np, g);
    } else {
      const RegN<S> rn = reg_n<S, T>(P.m.n, g);
      mont_mul<S, T>(a, bsh.p, bsh.s, rn, P.m.np, g);
    }
    __syncwarp();
    run_modexp<S, T>(a, P.e, P.m.n, P.m.np, tab, bsh, g);  // (r^n) R
    store_seg(A, a, g);
    __syncwarp();
    make_gm(GM, X, m64, mwide, e, P.nwords, Ln, L2, valid, status);
    grp_mont<L2, T>(X, A, GM, P.m.n, P.m.np, TT, g);  // r^n (1 + m n) mod n^2
    if (valid) write_tiled<T>(out, e, X, L2, g);
    __syncwarp();
  }
}

// ------------------------------------------------------------------ CRT decryption
template <int Lh, int T>
__device__ __forceinline__ void dec_half(const ModConst<Lh>& M, const Sched<kMaxSchedHalf>& E, const uint32_t* h,
                                         uint32_t hnp, const uint32_t* hinvlo, const uint32_t* hhR, const Col& X,
                                         const Col& OUT, const Col& A, const Col& B, const Col& C, const Col& TT,
                                         const Col& tab, const Col& bsh, const Grp<T>& g) {
  constexpr int S = Lh / T, Lp = Lh / 2;
  grp_to_mont_2l<Lh, T>(A, X, M.n, M.r2, M.r3, M.np, B, C, TT, g);  // c R mod h^2
  __syncwarp();
  uint32_t a[S];
  load_seg(a, A, g);
  run_modexp<S, T>(a, E, M.n, M.np, tab, bsh, g);          // c^(h-1) R mod h^2
  store_seg(A, a, g);
  __syncwarp();
  g_zero(B, Lh);
  B[0] = 1u;
  grp_mont<Lh, T>(C, A, B, M.n, M.np, TT, g);  // x = c^(h-1) mod h^2, x = 1 mod h
  // x - 1 (x >= 1)
  {
    uint64_t br = 1;
    for (int j = 0; j < Lh && br; ++j) {
      const uint32_t v = C[j];
      C[j] = v - 1u;
      br = (v == 0u);
    }
  }
  g_mul_lo(A, C, PArr{hinvlo}, Lp);   // L_h(x) = (x-1)/h exactly, via h^-1 mod 2^(32 Lp)
  grp_mont<Lp, T>(OUT, A, const_col(hhR), h, hnp, TT, g);  // m_h = L_h(x) h_h mod h
}

template <int Lh, int T>
__global__ void __launch_bounds__(kThreads, min_blocks(Lh, T)) k_dec_crt(const __grid_constant__ DecParams<Lh> P,
                                                      const uint32_t* __restrict__ ct, size_t count,
                                                      uint32_t* __restrict__ out, uint32_t* __restrict__ scratch,
                                                      int tabw, size_t ebase) {
  constexpr int Lp = Lh / 2;
  extern __shared__ uint32_t bsh_all[];
  const Grp<T> g;
  const Layout ly(T);
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
    for (int j = 0; j < 2 * Lh; ++j) X[j] = ct[tiled_index(ebase + e, j, 2 * Lh)];
    dec_half<Lh, T>(P.mp, P.ep, P.p, P.pnp, P.pinvlo, P.hpR, X, MP, A, B, C, TT, tab, bsh, g);
    dec_half<Lh, T>(P.mq, P.eq, P.q, P.qnp, P.qinvlo, P.hqR, X, MQ, A, B, C, TT, tab, bsh, g);
    // Garner: m = m_p + p [(m_q - m_p) p^-1 mod q]  (m_p < p < q)
    if (g_sub(A, MQ, MP, Lp)) g_add(A, A, PArr{P.q}, Lp);
    grp_mont<Lp, T>(C, A, const_col(P.pinvqR), P.q, P.qnp, TT, g);
    g_mul(X, C, Lp, PArr{P.p}, Lp);
    uint64_t c = 0;
    for (int j = 0; j < Lh; ++j) {
      c += (uint64_t)X[j] + (j < Lp ? MP[j] : 0u);
      X[j] = (uint32_t)c;
      c >>= 32;
    }
    if (valid) write_tiled<T>(out, ebase + e, X, Lh, g);
    __syncwarp();
  }
}

// ------------------------------------------------------------------ split CRT halves
// The results of k_enc_crt / k_dec_crt with the two CRT halves of an element
// computed at the same time: in a CTA the first half of the lane groups (two
// warps) works mod p^2 and the second half mod q^2 on the same elements, and
// the recombination follows a block barrier.  Each warp runs one exponent's
// schedule, so control flow stays uniform.  Halves the time per element when
// the batch leaves most of the GPU idle (small batches; any T, one lane per
// half included).
// Encryption also takes a second vector in the same launch: elements
// e >= P.split use r-stream kind2, counter e0 + (e - split) and tiled output
// position base2 + (e - split).
template <int Lh, int T>
__global__ void __launch_bounds__(kThreads, min_blocks(Lh, T)) k_enc_crt2(const __grid_constant__ EncCrtParams<Lh> P,
                                                      const uint64_t* __restrict__ m64,
                                                      const uint32_t* __restrict__ mwide, size_t count,
                                                      uint32_t* __restrict__ out, uint32_t* __restrict__ scratch,
                                                      int tabw, int* status, size_t base_out) {
  extern __shared__ uint32_t bsh_all[];
  const Grp<T> g;
  const Layout ly(T);
  const int H = ly.G / 2;  // elements per CTA and pass
  const int half = ly.gl >= H ? 1 : 0;
  const int pe = ly.gl - half * H;
  const Col bsh{bsh_all + ly.gl, ly.G};
  const Col tab = ly.slot(scratch, 0);
  const int SW = 2 * Lh + 4;
  const Col X = ly.slot(scratch, tabw + 0 * SW), GM = ly.slot(scratch, tabw + 1 * SW),
            A = ly.slot(scratch, tabw + 2 * SW), B = ly.slot(scratch, tabw + 3 * SW),
            C = ly.slot(scratch, tabw + 4 * SW), TT = ly.slot(scratch, tabw + 5 * SW),
            CH = ly.slot(scratch, tabw + 6 * SW);
  for (size_t base = (size_t)blockIdx.x * H; base < count; base += (size_t)gridDim.x * H) {
    size_t e = base + pe;
    const bool valid = e < count;
    if (!valid) e = count - 1;
    const bool second = e >= P.split;
    const size_t ei = second ? e - P.split : e;
    const uint32_t sid = P.round_ptr ? ((*P.round_ptr << 8) | (second ? P.kind2 : P.kind)) : P.stream;
    gen_r(X, P.seed, sid, P.e0 + ei, Lh + 2, 2 * Lh);
    make_gm(GM, A, m64, mwide, e, P.nwords, Lh, 2 * Lh, valid && half == 0, status);
    // the half is uniform per warp; each branch reads its constants at fixed offsets
    if (half) enc_half<Lh, T>(P.mq, P.eq, P.lq, X, GM, CH, A, B, C, TT, tab, bsh, g);
    else enc_half<Lh, T>(P.mp, P.ep, P.lp, X, GM, CH, A, B, C, TT, tab, bsh, g);
    __syncthreads();
    if (half == 0) {
      // Eq. (gA-C-B) with c_q from the partner group (gl + H) of this CTA
      const Col CP = CH, CQ{CH.p + H, CH.s};
      if (g_sub(A, CQ, CP, Lh)) g_add(A, A, PArr{P.mq.n}, Lh);
      grp_mont<Lh, T>(C, A, const_col(P.pinv2R), P.mq.n, P.mq.np, TT, g);
      g_mul(X, C, Lh, PArr{P.p2}, Lh);
      uint64_t c = 0;
      for (int j = 0; j < 2 * Lh; ++j) {
        c += (uint64_t)X[j] + (j < Lh ? CP[j] : 0u);
        X[j] = (uint32_t)c;
        c >>= 32;
      }
      if (valid) write_tiled<T>(out, (second ? P.base2 : base_out) + ei, X, 2 * Lh, g);
    }
    __syncthreads();
  }
}

template <int Lh, int T>
__global__ void __launch_bounds__(kThreads, min_blocks(Lh, T)) k_dec_crt2(const __grid_constant__ DecParams<Lh> P,
                                                      const uint32_t* __restrict__ ct, size_t count,
                                                      uint32_t* __restrict__ out, uint32_t* __restrict__ scratch,
                                                      int tabw, size_t ebase) {
  constexpr int Lp = Lh / 2;
  extern __shared__ uint32_t bsh_all[];
  const Grp<T> g;
  const Layout ly(T);
  const int H = ly.G / 2;
  const int half = ly.gl >= H ? 1 : 0;
  const int pe = ly.gl - half * H;
  const Col bsh{bsh_all + ly.gl, ly.G};
  const Col tab = ly.slot(scratch, 0);
  const int SW = 2 * Lh + 4;
  const Col X = ly.slot(scratch, tabw + 0 * SW), A = ly.slot(scratch, tabw + 1 * SW),
            B = ly.slot(scratch, tabw + 2 * SW), C = ly.slot(scratch, tabw + 3 * SW),
            TT = ly.slot(scratch, tabw + 4 * SW), MH = ly.slot(scratch, tabw + 5 * SW);
  for (size_t base = (size_t)blockIdx.x * H; base < count; base += (size_t)gridDim.x * H) {
    size_t e = base + pe;
    const bool valid = e < count;
    if (!valid) e = count - 1;
    for (int j = 0; j < 2 * Lh; ++j) X[j] = ct[tiled_index(ebase + e, j, 2 * Lh)];
    if (half) dec_half<Lh, T>(P.mq, P.eq, P.q, P.qnp, P.qinvlo, P.hqR, X, MH, A, B, C, TT, tab, bsh, g);
    else dec_half<Lh, T>(P.mp, P.ep, P.p, P.pnp, P.pinvlo, P.hpR, X, MH, A, B, C, TT, tab, bsh, g);
    __syncthreads();
    if (half == 0) {
      // Garner: m = m_p + p [(m_q - m_p) p^-1 mod q], m_q from the partner group
      const Col MP = MH, MQ{MH.p + H, MH.s};
      if (g_sub(A, MQ, MP, Lp)) g_add(A, A, PArr{P.q}, Lp);
      grp_mont<Lp, T>(C, A, const_col(P.pinvqR), P.q, P.qnp, TT, g);
      g_mul(X, C, Lp, PArr{P.p}, Lp);
      uint64_t c = 0;
      for (int j = 0; j < Lh; ++j) {
        c += (uint64_t)X[j] + (j < Lp ? MP[j] : 0u);
        X[j] = (uint32_t)c;
        c >>= 32;
      }
      if (valid) write_tiled<T>(out, ebase + e, X, Lh, g);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ homomorphic ops
template <int L2, int T>
__global__ void __launch_bounds__(kThreads, min_blocks(L2, T)) k_hom_sum(const __grid_constant__ HomParams<L2> P, size_t count,
                                                      uint32_t* __restrict__ out, size_t ebase) {
  constexpr int S = L2 / T;
  extern __shared__ uint32_t bsh_all[];
  const Grp<T> g;
  const Layout ly(T);
  const Col bsh{bsh_all + ly.gl, ly.G};
  RegN<S> rn;
  if constexpr (T > 1) rn = reg_n<S, T>(P.m.n, g);
  for (size_t base = (size_t)blockIdx.x * ly.G; base < count; base += (size_t)ly.Gtot) {
    size_t e = base + ly.gl;
    const bool valid = e < count;
    if (!valid) e = count - 1;
    uint32_t a[S];
#pragma unroll
    for (int j = 0; j < S; ++j) a[j] = P.src[0][tiled_index(ebase + e, g.k * S + j, L2)];
    for (int op = 1; op <= P.ngroups; ++op) {
      // operands 1..ngroups-1, then the fix-up factor R^k
      if (op < P.ngroups) {
        const uint32_t* src = P.src[op];
#pragma unroll
        for (int j = 0; j < S; ++j) bsh[g.k * S + j] = src[tiled_index(ebase + e, g.k * S + j, L2)];
      } else {
#pragma unroll
        for (int j = 0; j < S; ++j) bsh[g.k * S + j] = P.rk[g.k * S + j];
      }
      __syncwarp();
      if constexpr (T == 1) mont_mul<S, T>(a, bsh.p, bsh.s, ParamN{P.m.n}, P.m.np, g);
      else mont_mul<S, T>(a, bsh.p, bsh.s, rn, P.m.np, g);
      __syncwarp();
    }
    if (valid) {
#pragma unroll
      for (int j = 0; j < S; ++j) out[tiled_index(ebase + e, g.k * S + j, L2)] = a[j];
    }
  }
}

template <int L2, int T>
__global__ void __launch_bounds__(kThreads, min_blocks(L2, T)) k_hom_scal(const __grid_constant__ HomParams<L2> P,
                                                       const uint32_t* __restrict__ ct,
                                                       const uint64_t* __restrict__ kvec, size_t count,
                                                       uint32_t* __restrict__ out, uint32_t* __restrict__ scratch) {
  constexpr int S = L2 / T;
  extern __shared__ uint32_t bsh_all[];
  const Grp<T> g;
  const Layout ly(T);
  const Col bsh{bsh_all + ly.gl, ly.G};
  const Col tab = ly.slot(scratch, 0);
  RegN<S> rn;
  if constexpr (T > 1) rn = reg_n<S, T>(P.m.n, g);
  for (size_t base = (size_t)blockIdx.x * ly.G; base < count; base += (size_t)ly.Gtot) {
    size_t e = base + ly.gl;
    const bool valid = e < count;
    if (!valid) e = count - 1;
    uint32_t a[S];
#pragma unroll
    for (int j = 0; j < S; ++j) a[j] = ct[tiled_index(e, g.k * S + j, L2)];
#pragma unroll
    for (int j = 0; j < S; ++j) bsh[g.k * S + j] = P.m.r2[g.k * S + j];
    __syncwarp();
    if constexpr (T == 1) mont_mul<S, T>(a, bsh.p, bsh.s, ParamN{P.m.n}, P.m.np, g);
    else mont_mul<S, T>(a, bsh.p, bsh.s, rn, P.m.np, g);
    __syncwarp();
    const uint64_t k = kvec[e];
    // digits needed by the widest exponent of the warp (uniform)
    const uint32_t hi = __reduce_or_sync(PC2_FULL, (uint32_t)(k >> 32));
    const uint32_t lo = __reduce_or_sync(PC2_FULL, (uint32_t)k);
    const int bits = hi ? 64 - __clz(hi) : (lo ? 32 - __clz(lo) : 1);
    const int nd = (bits + P.w - 1) / P.w;
    if constexpr (T == 1) modexp_var<S, T>(a, k, P.w, nd, P.m.r1, tab, bsh, ParamN{P.m.n}, P.m.np, g);
    else modexp_var<S, T>(a, k, P.w, nd, P.m.r1, tab, bsh, rn, P.m.np, g);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < S; ++j) bsh[g.k * S + j] = (g.k == 0 && j == 0) ? 1u : 0u;
    __syncwarp();
    if constexpr (T == 1) mont_mul<S, T>(a, bsh.p, bsh.s, ParamN{P.m.n}, P.m.np, g);
    else mont_mul<S, T>(a, bsh.p, bsh.s, rn, P.m.np, g);
    __syncwarp();
    if (valid) {
#pragma unroll
      for (int j = 0; j < S; ++j) out[tiled_index(e, g.k * S + j, L2)] = a[j];
    }
  }
}

// Definition 2 with a full-width scalar: c^k mod n^2 for a per-element k of
// Lk = L2 / 2 words (tiled input).  Fixed windows of P.w bits over all Lk
// words, the same number of digits for every element.
template <int L2, int T>
__global__ void __launch_bounds__(kThreads, min_blocks(L2, T)) k_hom_scal_wide(const __grid_constant__ HomParams<L2> P,
                                                       const uint32_t* __restrict__ ct,
                                                       const uint32_t* __restrict__ kw, size_t count,
                                                       uint32_t* __restrict__ out, uint32_t* __restrict__ scratch) {
  constexpr int S = L2 / T, Lk = L2 / 2;
  extern __shared__ uint32_t bsh_all[];
  const Grp<T> g;
  const Layout ly(T);
  const Col bsh{bsh_all + ly.gl, ly.G};
  const Col tab = ly.slot(scratch, 0);
  RegN<S> rn;
  if constexpr (T > 1) rn = reg_n<S, T>(P.m.n, g);
  const int w = P.w;
  const uint32_t mask = (1u << w) - 1u;
  const int nd = (32 * Lk + w - 1) / w;
  for (size_t base = (size_t)blockIdx.x * ly.G; base < count; base += (size_t)ly.Gtot) {
    size_t e = base + ly.gl;
    const bool valid = e < count;
    if (!valid) e = count - 1;
    uint32_t a[S];
#pragma unroll
    for (int j = 0; j < S; ++j) a[j] = ct[tiled_index(e, g.k * S + j, L2)];
#pragma unroll
    for (int j = 0; j < S; ++j) bsh[g.k * S + j] = P.m.r2[g.k * S + j];
    __syncwarp();
    if constexpr (T == 1) mont_mul<S, T>(a, bsh.p, bsh.s, ParamN{P.m.n}, P.m.np, g);
    else mont_mul<S, T>(a, bsh.p, bsh.s, rn, P.m.np, g);
    __syncwarp();
    // digit pos: bits [pos w, pos w + w) of k, read across a word boundary when needed
    auto digit = [&](int pos) {
      const int b0 = pos * w, wi = b0 >> 5, sh = b0 & 31;
      uint64_t v = kw[tiled_index(e, wi, Lk)];
      if (wi + 1 < Lk) v |= (uint64_t)kw[tiled_index(e, wi + 1, Lk)] << 32;
      return (int)((uint32_t)(v >> sh) & mask);
    };
    if constexpr (T == 1) modexp_digits<S, T>(a, digit, w, nd, P.m.r1, tab, bsh, ParamN{P.m.n}, P.m.np, g);
    else modexp_digits<S, T>(a, digit, w, nd, P.m.r1, tab, bsh, rn, P.m.np, g);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < S; ++j) bsh[g.k * S + j] = (g.k == 0 && j == 0) ? 1u : 0u;
    __syncwarp();
    if constexpr (T == 1) mont_mul<S, T>(a, bsh.p, bsh.s, ParamN{P.m.n}, P.m.np, g);
    else mont_mul<S, T>(a, bsh.p, bsh.s, rn, P.m.np, g);
    __syncwarp();
    if (valid) {
#pragma unroll
      for (int j = 0; j < S; ++j) out[tiled_index(e, g.k * S + j, L2)] = a[j];
    }
  }
}

}  // namespace pc2
