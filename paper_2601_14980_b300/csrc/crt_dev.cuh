// crt_dev.cuh -- per-element device steps shared by the persistent
// multi-request kernels (the batched ADMM round and the serving steps):
// g^m = 1 + m n, one CRT half of an encryption (Eq. (itq1) mod p^2 or q^2,
// Sec. IV-A) and of a decryption (Sec. III-C, L_p(c^(p-1) mod p^2) h_p), and
// a fixed-window power on the word-serial glue.
#pragma once
#include <cuda_runtime.h>

#include "paillier_kernels.cuh"

namespace pc2 {

// GM = 1 + m n for a 64-bit m (zero-padded to `total` words); M: temporary column.
__device__ __forceinline__ void gm_u64(const Col& GM, const Col& M, uint64_t m, const uint32_t* n, int Ln, int total) {
  M[0] = (uint32_t)m;
  M[1] = (uint32_t)(m >> 32);
  g_mul(GM, M, 2, PArr{n}, Ln);
  uint64_t c = 1;
  for (int j = 0; j < 2 + Ln; ++j) {
    c += GM[j];
    GM[j] = (uint32_t)c;
    c >>= 32;
  }
  for (int j = 2 + Ln; j < total; ++j) GM[j] = 0u;
}

// One CRT half of an encryption: OUT = r^n (1 + m n) mod h^2 (h^2 = Mg.n).
// Mg, Hg: the half's constants in device memory; nfast, hfast: h^2 and h in
// constant memory (read with compile-time offsets by one-lane products; with
// T > 1 each lane loads its segment of Mg.n, Hg.h.n into registers instead).
// r^n mod h^2 takes the lifted route (LiftConst) where a lane holds at least
// two half-width limbs, else the power by n mod h(h-1) (schedule E).
template <int Lh, int T, int MaxS = 64>
__device__ __forceinline__ void enc_half_f(const ModConst<Lh>& Mg, const uint32_t* nfast, const Sched<kMaxSched>& E,
                                           const LiftConst<Lh>& Hg, const uint32_t* hfast, const Col& X,
                                           const Col& GM, const Col& OUT, const Col& A, const Col& B, const Col& C,
                                           const Col& TT, const Col& tab, const Col& bsh, const Grp<T>& g) {
  constexpr int S = Lh / T;
  const uint32_t np = Mg.np;
  if constexpr (lift_route<Lh, T>()) {
    rn_lifted<Lh, T>(Mg, nfast, Hg, hfast, X, A, B, C, TT, tab, bsh, g);  // (r^n mod h^2) R
  } else {
    grp_to_mont_2l<Lh, T, MaxS>(A, X, Mg.n, Mg.r2, Mg.r3, np, B, C, TT, g);  // r R mod h^2
    __syncwarp();
    uint32_t a[S];
    load_seg(a, A, g);
    if constexpr (T == 1) run_modexp<S, T>(a, E, nfast, np, tab, bsh, g);
    else run_modexp<S, T>(a, E, Mg.n, np, tab, bsh, g);      // (r^n mod h^2) R
    store_seg(A, a, g);
    __syncwarp();
  }
  grp_to_mont_2l<Lh, T, MaxS>(B, GM, Mg.n, Mg.r2, Mg.r3, np, C, OUT, TT, g);  // (1 + m n) R mod h^2
  grp_mont<Lh, T, MaxS>(C, A, B, Mg.n, np, TT, g);
  g_zero(B, Lh);
  B[0] = 1u;
  grp_mont<Lh, T, MaxS>(OUT, C, B, Mg.n, np, TT, g);
}

// One CRT half of a decryption: OUT = L_h(c^(h-1) mod h^2) h_h mod h.
template <int Lh, int T, int MaxS = 64>
__device__ __forceinline__ void dec_half_f(const ModConst<Lh>& Mg, const uint32_t* nfast,
                                           const Sched<kMaxSchedHalf>& E, const uint32_t* h,
                                           uint32_t hnp, const uint32_t* hinvlo, const uint32_t* hhR, const Col& X,
                                           const Col& OUT, const Col& A, const Col& B, const Col& C, const Col& TT,
                                           const Col& tab, const Col& bsh, const Grp<T>& g) {
  constexpr int S = Lh / T, Lp = Lh / 2;
  const uint32_t np = Mg.np;
  grp_to_mont_2l<Lh, T, MaxS>(A, X, Mg.n, Mg.r2, Mg.r3, np, B, C, TT, g);  // c R mod h^2
  __syncwarp();
  uint32_t a[S];
  load_seg(a, A, g);
  if constexpr (T == 1) run_modexp<S, T>(a, E, nfast, np, tab, bsh, g);
  else run_modexp<S, T>(a, E, Mg.n, np, tab, bsh, g);      // c^(h-1) R mod h^2
  store_seg(A, a, g);
  __syncwarp();
  g_zero(B, Lh);
  B[0] = 1u;
  grp_mont<Lh, T, MaxS>(C, A, B, Mg.n, np, TT, g);  // x = c^(h-1) mod h^2 = 1 mod h
  {
    uint64_t br = 1;
    for (int j = 0; j < Lh && br; ++j) {
      const uint32_t v = C[j];
      C[j] = v - 1u;
      br = (v == 0u);
    }
  }
  g_mul_lo(A, C, PArr{hinvlo}, Lp);  // (x - 1) / h exactly
  grp_mont<Lp, T, MaxS>(OUT, A, const_col(hhR), h, hnp, TT, g);
}

// acc = base^k in Montgomery form (base given as x R), fixed windows of w
// bits over nd digits (warp-uniform); tab: 2^w entries of L words.  The
// products go through the lane group (grp_mont).
template <int L, int T, int MaxS = 64>
__device__ __forceinline__ void grp_pow_u64(const Col& acc, const Col& base, uint64_t k, int w, int nd, const Col& tab,
                                            const uint32_t* r1, const uint32_t* N, uint32_t np, const Col& tt,
                                            const Grp<T>& g) {
  const int ntab = 1 << w;
  const uint64_t mask = (uint64_t)ntab - 1u;
  g_copy_param(tab, r1, L);
  g_copy(tab.off(L), base, L);
  for (int d = 2; d < ntab; ++d) grp_mont<L, T, MaxS>(tab.off(d * L), tab.off((d - 1) * L), tab.off(L), N, np, tt, g);
  int pos = nd - 1;
  g_copy(acc, tab.off((int)((k >> (pos * w)) & mask) * L), L);
  for (--pos; pos >= 0; --pos) {
    for (int s = 0; s < w; ++s) grp_mont<L, T, MaxS>(acc, acc, acc, N, np, tt, g);
    grp_mont<L, T, MaxS>(acc, acc, tab.off((int)((k >> (pos * w)) & mask) * L), N, np, tt, g);
  }
}

constexpr int kScalWin = 4;  // window of a scaling exponent (< 2^64) on the glue

}  // namespace pc2
