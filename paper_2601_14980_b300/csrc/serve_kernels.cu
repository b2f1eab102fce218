// serve_kernels.cu -- one step of the serving loop: a persistent launch over
// the work items of every active request, whatever its operation.
//
//   encrypt    Eq. (itq1) through the CRT split of Sec. IV-A (the server owns
//              the key), r as pc2_encrypt draws it (stream, counter e0 + i)
//   decrypt    Sec. III-C through the CRT (L_p(c^(p-1) mod p^2) h_p, Garner)
//   aggregate  Definition 1 over `groups` operand vectors: prod_g c_g mod n^2
//
// Each step gives every element one lane when the step's work fills the GPU,
// else one, two or eight lanes per CRT half with the two halves in parallel
// (shorter latency per element when the GPU would idle).  Every result is the
// one the per-operation entry points compute (pc2_encrypt, pc2_decrypt,
// pc2_hom_sum), whatever else runs in the same step.
#include <cuda_runtime.h>

#include "crt_dev.cuh"
#include "pc2_serve.h"

namespace pc2 {

__constant__ ServeConst<16> c_serve16;
__constant__ ServeConst<64> c_serve64;

template <int Lh>
__device__ __forceinline__ const ServeConst<Lh>& serve_const() {
  if constexpr (Lh == 16) return c_serve16;
  else return c_serve64;
}

// Element slots of the CTA-local scratch for `G` groups.
struct CtaCols {
  uint32_t* base;
  int G, gl;
  __device__ __forceinline__ Col row(int r) const { return Col{base + (size_t)r * G + gl, G}; }
};

template <int Lh, int T>
__device__ __forceinline__ void serve_encrypt(const ServeKey<Lh>& K, const ServeReq& R, const ServeItem& I, int tabw,
                                              uint32_t* cta, uint32_t* bsh_all, int* status) {
  constexpr int L2 = 2 * Lh, G = kThreads / T;
  const Grp<T> g;
  const CtaCols cc{cta, G, (int)threadIdx.x / T};
  const Col bsh{bsh_all + cc.gl, G};
  const int SW = L2 + 4;
  const Col tab = cc.row(0), X = cc.row(tabw), GM = cc.row(tabw + SW), A = cc.row(tabw + 2 * SW),
            B = cc.row(tabw + 3 * SW), C = cc.row(tabw + 4 * SW), TT = cc.row(tabw + 5 * SW),
            CP = cc.row(tabw + 6 * SW), CQ = cc.row(tabw + 7 * SW);
  const bool valid = cc.gl < (int)I.count;
  const size_t idx = I.first + (valid ? (uint32_t)cc.gl : I.count - 1u);
  gen_r(X, R.seed, R.stream, R.e0 + idx, Lh + 2, L2);
  gm_u64(GM, A, R.m64[idx], K.enc.nwords, Lh, L2);
  enc_half_f<Lh, T>(K.enc.mp, serve_const<Lh>().mp, K.enc.ep, K.enc.lp, serve_const<Lh>().hp, X, GM, CP, A, B, C, TT, tab, bsh, g);
  enc_half_f<Lh, T>(K.enc.mq, serve_const<Lh>().mq, K.enc.eq, K.enc.lq, serve_const<Lh>().hq, X, GM, CQ, A, B, C, TT, tab, bsh, g);
  // Eq. (gA-C-B): c = c_p + [(c_q - c_p) (p^2)^-1 mod q^2] p^2
  if (g_sub(A, CQ, CP, Lh)) g_add(A, A, PArr{K.enc.mq.n}, Lh);
  grp_mont<Lh, T>(C, A, const_col(K.enc.pinv2R), K.enc.mq.n, K.enc.mq.np, TT, g);
  g_mul(X, C, Lh, PArr{K.enc.p2}, Lh);
  uint64_t c = 0;
  for (int j = 0; j < L2; ++j) {
    c += (uint64_t)X[j] + (j < Lh ? CP[j] : 0u);
    X[j] = (uint32_t)c;
    c >>= 32;
  }
  if (valid) write_tiled<T>(R.out, idx, X, L2, g);
  __syncwarp();
  (void)status;
}

template <int Lh, int T>
__device__ __forceinline__ void serve_decrypt(const ServeKey<Lh>& K, const ServeReq& R, const ServeItem& I, int tabw,
                                              uint32_t* cta, uint32_t* bsh_all) {
  constexpr int L2 = 2 * Lh, Lp = Lh / 2, G = kThreads / T;
  const Grp<T> g;
  const CtaCols cc{cta, G, (int)threadIdx.x / T};
  const Col bsh{bsh_all + cc.gl, G};
  const int SW = L2 + 4;
  const Col tab = cc.row(0), X = cc.row(tabw), A = cc.row(tabw + SW), B = cc.row(tabw + 2 * SW),
            C = cc.row(tabw + 3 * SW), TT = cc.row(tabw + 4 * SW), MP = cc.row(tabw + 5 * SW),
            MQ = cc.row(tabw + 6 * SW);
  const bool valid = cc.gl < (int)I.count;
  const size_t idx = I.first + (valid ? (uint32_t)cc.gl : I.count - 1u);
  for (int j = 0; j < L2; ++j) X[j] = R.ct_in[tiled_index(idx, j, L2)];
  dec_half_f<Lh, T>(K.dec.mp, serve_const<Lh>().mp, K.dec.ep, K.dec.p, K.dec.pnp, K.dec.pinvlo, K.dec.hpR, X, MP, A,
                    B, C, TT, tab, bsh, g);
  dec_half_f<Lh, T>(K.dec.mq, serve_const<Lh>().mq, K.dec.eq, K.dec.q, K.dec.qnp, K.dec.qinvlo, K.dec.hqR, X, MQ, A,
                    B, C, TT, tab, bsh, g);
  // Garner: m = m_p + p [(m_q - m_p) p^-1 mod q]
  if (g_sub(A, MQ, MP, Lp)) g_add(A, A, PArr{K.dec.q}, Lp);
  grp_mont<Lp, T>(C, A, const_col(K.dec.pinvqR), K.dec.q, K.dec.qnp, TT, g);
  g_mul(X, C, Lp, PArr{K.dec.p}, Lp);
  uint64_t c = 0;
  for (int j = 0; j < Lh; ++j) {
    c += (uint64_t)X[j] + (j < Lp ? MP[j] : 0u);
    X[j] = (uint32_t)c;
    c >>= 32;
  }
  if (valid) write_tiled<T>(R.out, idx, X, Lh, g);
  __syncwarp();
}

// Small requests: the two CRT halves of each element in parallel (the first
// two warps mod p^2, the last two mod q^2, same elements), recombined after a
// block barrier; the CTA takes 64 / T elements per item.
template <int Lh, int T>
__device__ __forceinline__ void serve_encrypt_split(const ServeKey<Lh>& K, const ServeReq& R, const ServeItem& I,
                                                    int tabw, uint32_t* cta, uint32_t* bsh_all) {
  constexpr int L2 = 2 * Lh, G = kThreads / T, H = G / 2;
  const Grp<T> g;
  const CtaCols cc{cta, G, (int)threadIdx.x / T};
  const int half = cc.gl >= H ? 1 : 0, pe = cc.gl - half * H;
  const Col bsh{bsh_all + cc.gl, G};
  const int SW = L2 + 4;
  const Col tab = cc.row(0), X = cc.row(tabw), GM = cc.row(tabw + SW), A = cc.row(tabw + 2 * SW),
            B = cc.row(tabw + 3 * SW), C = cc.row(tabw + 4 * SW), TT = cc.row(tabw + 5 * SW),
            CH = cc.row(tabw + 6 * SW);
  const bool valid = pe < (int)I.count;
  const size_t idx = I.first + (valid ? (uint32_t)pe : I.count - 1u);
  gen_r(X, R.seed, R.stream, R.e0 + idx, Lh + 2, L2);
  gm_u64(GM, A, R.m64[idx], K.enc.nwords, Lh, L2);
  if (half) enc_half_f<Lh, T>(K.enc.mq, serve_const<Lh>().mq, K.enc.eq, K.enc.lq, serve_const<Lh>().hq, X, GM, CH, A, B, C, TT, tab, bsh, g);
  else enc_half_f<Lh, T>(K.enc.mp, serve_const<Lh>().mp, K.enc.ep, K.enc.lp, serve_const<Lh>().hp, X, GM, CH, A, B, C, TT, tab, bsh, g);
  __syncthreads();
  if (!half) {
    const Col CP = CH, CQ{CH.p + H, CH.s};
    if (g_sub(A, CQ, CP, Lh)) g_add(A, A, PArr{K.enc.mq.n}, Lh);
    grp_mont<Lh, T>(C, A, const_col(K.enc.pinv2R), K.enc.mq.n, K.enc.mq.np, TT, g);
    g_mul(X, C, Lh, PArr{K.enc.p2}, Lh);
    uint64_t c = 0;
    for (int j = 0; j < L2; ++j) {
      c += (uint64_t)X[j] + (j < Lh ? CP[j] : 0u);
      X[j] = (uint32_t)c;
      c >>= 32;
    }
    if (valid) write_tiled<T>(R.out, idx, X, L2, g);
  }
  __syncthreads();
}

template <int Lh, int T>
__device__ __forceinline__ void serve_decrypt_split(const ServeKey<Lh>& K, const ServeReq& R, const ServeItem& I,
                                                    int tabw, uint32_t* cta, uint32_t* bsh_all) {
  constexpr int L2 = 2 * Lh, Lp = Lh / 2, G = kThreads / T, H = G / 2;
  const Grp<T> g;
  const CtaCols cc{cta, G, (int)threadIdx.x / T};
  const int half = cc.gl >= H ? 1 : 0, pe = cc.gl - half * H;
  const Col bsh{bsh_all + cc.gl, G};
  const int SW = L2 + 4;
  const Col tab = cc.row(0), X = cc.row(tabw), A = cc.row(tabw + SW), B = cc.row(tabw + 2 * SW),
            C = cc.row(tabw + 3 * SW), TT = cc.row(tabw + 4 * SW), MH = cc.row(tabw + 5 * SW);
  const bool valid = pe < (int)I.count;
  const size_t idx = I.first + (valid ? (uint32_t)pe : I.count - 1u);
  for (int j = 0; j < L2; ++j) X[j] = R.ct_in[tiled_index(idx, j, L2)];
  if (half)
    dec_half_f<Lh, T>(K.dec.mq, serve_const<Lh>().mq, K.dec.eq, K.dec.q, K.dec.qnp, K.dec.qinvlo, K.dec.hqR, X, MH,
                      A, B, C, TT, tab, bsh, g);
  else
    dec_half_f<Lh, T>(K.dec.mp, serve_const<Lh>().mp, K.dec.ep, K.dec.p, K.dec.pnp, K.dec.pinvlo, K.dec.hpR, X, MH,
                      A, B, C, TT, tab, bsh, g);
  __syncthreads();
  if (!half) {
    const Col MP = MH, MQ{MH.p + H, MH.s};
    if (g_sub(A, MQ, MP, Lp)) g_add(A, A, PArr{K.dec.q}, Lp);
    grp_mont<Lp, T>(C, A, const_col(K.dec.pinvqR), K.dec.q, K.dec.qnp, TT, g);
    g_mul(X, C, Lp, PArr{K.dec.p}, Lp);
    uint64_t c = 0;
    for (int j = 0; j < Lh; ++j) {
      c += (uint64_t)X[j] + (j < Lp ? MP[j] : 0u);
      X[j] = (uint32_t)c;
      c >>= 32;
    }
    if (valid) write_tiled<T>(R.out, idx, X, Lh, g);
  }
  __syncthreads();
}

// prod_g c_g mod n^2: g - 1 Montgomery products, then the fix-up R^groups.
template <int Lh>
__device__ __forceinline__ void serve_aggregate(const ServeKey<Lh>& K, const ServeReq& R, const ServeItem& I,
                                                uint32_t* bsh_all) {
  constexpr int L2 = 2 * Lh, T = serve_agg_lanes(L2), S = L2 / T, G = kThreads / T;
  const Grp<T> g;
  const int gl = (int)threadIdx.x / T;
  const Col bsh{bsh_all + gl, G};
  const bool valid = gl < (int)I.count;
  const size_t idx = I.first + (valid ? (uint32_t)gl : I.count - 1u);
  RegN<S> rn;
  if constexpr (T > 1) rn = reg_n<S, T>(K.n2.n, g);
  const uint32_t np = K.n2.np;
  uint32_t a[S];
#pragma unroll
  for (int j = 0; j < S; ++j) a[j] = R.ct_in[tiled_index(idx, g.k * S + j, L2)];
  const int ng = (int)R.groups;
  for (int op = 1; op <= ng; ++op) {
    if (op < ng) {
      const uint32_t* src = R.ct_in + (size_t)op * R.ct_stride;
#pragma unroll
      for (int j = 0; j < S; ++j) bsh[g.k * S + j] = src[tiled_index(idx, g.k * S + j, L2)];
    } else {
#pragma unroll
      for (int j = 0; j < S; ++j) bsh[g.k * S + j] = K.rpow[ng][g.k * S + j];
    }
    __syncwarp();
    if constexpr (T == 1) mont_mul<S, T>(a, bsh.p, bsh.s, ParamN{serve_const<Lh>().n2}, np, g);
    else mont_mul<S, T>(a, bsh.p, bsh.s, rn, np, g);
    __syncwarp();
  }
  if (valid) {
#pragma unroll
    for (int j = 0; j < S; ++j) R.out[tiled_index(idx, g.k * S + j, L2)] = a[j];
  }
}

template <int Lh>
__global__ void __launch_bounds__(kThreads, 3) k_serve_step(const __grid_constant__ ServeParams P) {
  extern __shared__ uint32_t bsh_all[];
  __shared__ uint32_t s_item;
  const ServeKey<Lh>& K = *static_cast<const ServeKey<Lh>*>(P.key);
  uint32_t* cta = P.scratch + (size_t)blockIdx.x * P.cta_words;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(P.next, 1u);
    __syncthreads();
    const uint32_t it = s_item;
    __syncthreads();
    if (it >= P.nitems) break;
    const ServeItem I = P.items[it];
    const ServeReq& R = P.reqs[I.req];
    switch (I.kind) {
      case SK_ENC1: serve_encrypt<Lh, 1>(K, R, I, P.tabw, cta, bsh_all, P.status); break;
      case SK_ENC8: serve_encrypt_split<Lh, kServeLanesSmall>(K, R, I, P.tabw, cta, bsh_all); break;
      case SK_DEC1: serve_decrypt<Lh, 1>(K, R, I, P.tabw, cta, bsh_all); break;
      case SK_DEC8: serve_decrypt_split<Lh, kServeLanesSmall>(K, R, I, P.tabw, cta, bsh_all); break;
      case SK_AGG: serve_aggregate<Lh>(K, R, I, bsh_all); break;
      case SK_ENC2: serve_encrypt_split<Lh, 2>(K, R, I, P.tabw, cta, bsh_all); break;
      case SK_DEC2: serve_decrypt_split<Lh, 2>(K, R, I, P.tabw, cta, bsh_all); break;
      default: break;
    }
  }
}

// The one-lane-per-half items (SK_ENC1S, SK_DEC1S) in a kernel of their own:
// inside k_serve_step their two 64-limb copies of the exponentiation next to
// the other item kinds raised the register pressure of the whole kernel into
// heavy spilling.
template <int Lh>
__global__ void __launch_bounds__(kThreads, 3) k_serve_step_s1(const __grid_constant__ ServeParams P) {
  extern __shared__ uint32_t bsh_all[];
  __shared__ uint32_t s_item;
  const ServeKey<Lh>& K = *static_cast<const ServeKey<Lh>*>(P.key);
  uint32_t* cta = P.scratch + (size_t)blockIdx.x * P.cta_words;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(P.next, 1u);
    __syncthreads();
    const uint32_t it = s_item;
    __syncthreads();
    if (it >= P.nitems) break;
    const ServeItem I = P.items[it];
    const ServeReq& R = P.reqs[I.req];
    if (I.kind == SK_ENC1S) serve_encrypt_split<Lh, 1>(K, R, I, P.tabw, cta, bsh_all);
    else if (I.kind == SK_DEC1S) serve_decrypt_split<Lh, 1>(K, R, I, P.tabw, cta, bsh_all);
  }
}

template <int Lh>
int serve_blocks_per_sm(size_t smem) {
  int per = 0;
  if (cudaFuncSetAttribute(k_serve_step<Lh>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_serve_step<Lh>, kThreads, smem) != cudaSuccess) return -1;
  return per;
}

template <int Lh>
int serve_set_const(const ServeConst<Lh>* d_const, cudaStream_t st) {
  const void* sym = nullptr;
  if constexpr (Lh == 16) sym = (const void*)&c_serve16;
  else sym = (const void*)&c_serve64;
  if (cudaMemcpyToSymbolAsync(sym, d_const, sizeof(ServeConst<Lh>), 0, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return PC2_ECUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

template <int Lh>
int launch_serve_step(const ServeParams& P, size_t smem, int grid, cudaStream_t st, bool one_lane_split) {
  if (one_lane_split) {
    if (cudaFuncSetAttribute(k_serve_step_s1<Lh>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return PC2_ECUDA;
    k_serve_step_s1<Lh><<<grid, kThreads, smem, st>>>(P);
  } else {
    k_serve_step<Lh><<<grid, kThreads, smem, st>>>(P);
  }
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

template int launch_serve_step<16>(const ServeParams&, size_t, int, cudaStream_t, bool);
template int launch_serve_step<64>(const ServeParams&, size_t, int, cudaStream_t, bool);
template int serve_set_const<16>(const ServeConst<16>*, cudaStream_t);
template int serve_set_const<64>(const ServeConst<64>*, cudaStream_t);
template int serve_blocks_per_sm<16>(size_t);
template int serve_blocks_per_sm<64>(size_t);

}  // namespace pc2
