// batch_kernels.cu -- the batched private ADMM round: one persistent launch
// runs the whole round of every element of every edge node in its work list,
// whatever the node's key size (pc2_batch.h states the element-wise form of
// the round; the host leaves out the nodes it runs on the tensor cores).
//
//   k_batch_round   persistent CTAs claim work items (up to 128 / lanes
//                   consecutive elements of one node) from a cost-ordered
//                   list; per element: Gamma2(z), Gamma2(-v) (Eq. (et21));
//                   two CRT encryptions (Eq. (itq1), Sec. IV-A, Lemmas 1-2);
//                   s-hat = z-hat (+) (-v)-hat (Definition 1); x-hat =
//                   alpha-hat (+) b (x) s-hat (Definition 2, Eq. (itq2));
//                   CRT decryption (Sec. III-C); the exact decode of Theorem 1
//                   (N_k = 1); z = S_kappa(v + x), v = v + x - z (Eqs. (ty32),
//                   (u78)).  The last CTA to finish advances the round counter
//                   and re-arms the work list, so a captured launch replays
//                   round after round.
//   k_batch_update  the decode and z/v update alone, for the plain per-node
//                   path (which runs the other steps through the library's
//                   per-operation kernels).
//
// The modular exponentiations run on the register Montgomery core (mont.cuh)
// with the CRT moduli of one-lane classes in constant memory; the few other
// Montgomery products per element (CRT recombination, aggregation, the
// 28-bit scaling exponent, the product with alpha-hat) run in the lane
// group's registers where a lane holds at most 32 words, else on the
// word-serial glue.
#include <cuda_runtime.h>

#include "admm_dev.cuh"
#include "crt_dev.cuh"
#include "pc2_batch.h"

namespace pc2 {

__constant__ BatchConstMods c_bmods;

// Modulus of CRT half H (0: p^2, 1: q^2) of a one-lane class, in constant memory.
template <int Lh, int H>
__device__ __forceinline__ const uint32_t* bmod() {
  if constexpr (Lh == 8) return c_bmods.m8[H];
  else if constexpr (Lh == 16) return c_bmods.m16[H];
  else if constexpr (Lh == 32) return c_bmods.m32[H];
  else if constexpr (Lh == 64) return c_bmods.m64[H];
  else return nullptr;
}

// Prime of CRT half H (0: p, 1: q) of a one-lane class, in constant memory.
template <int Lh, int H>
__device__ __forceinline__ const uint32_t* bprime() {
  if constexpr (Lh == 8) return c_bmods.h8[H];
  else if constexpr (Lh == 16) return c_bmods.h16[H];
  else if constexpr (Lh == 32) return c_bmods.h32[H];
  else if constexpr (Lh == 64) return c_bmods.h64[H];
  else return nullptr;
}

template <int Lh, int T>
__device__ __forceinline__ void batch_item(const BatchParams& P, const BatchItem& I, uint32_t round, uint32_t* cta,
                                           uint32_t* bsh_all) {
  constexpr int L2 = 2 * Lh, Lp = Lh / 2, G = kThreads / T;
  constexpr int cls = batch_class(Lh);
  // glue products in registers up to 32 words per lane: the one kernel holds
  // every key class under one register budget, and wider segments spill
  constexpr int MS = 32;
  const Grp<T> g;
  const int gl = (int)threadIdx.x / T;
  const BatchKey<Lh>& K = *static_cast<const BatchKey<Lh>*>(P.key[cls]);
  const BatchNode nd = P.nodes[I.node];
  const int tabw = P.tabw[cls];
  const int SW = L2 + 4;
  auto slot = [&](int row) { return Col{cta + (size_t)row * G + gl, G}; };
  const Col bsh{bsh_all + gl, G};
  const Col tab = slot(0);
  const Col X = slot(tabw), GM = slot(tabw + SW), A = slot(tabw + 2 * SW), B = slot(tabw + 3 * SW),
            C = slot(tabw + 4 * SW), TT = slot(tabw + 5 * SW), CP = slot(tabw + 6 * SW), CQ = slot(tabw + 7 * SW),
            CZ = slot(tabw + 8 * SW), CV = slot(tabw + 9 * SW);
  const bool valid = gl < (int)I.count;
  const uint32_t idx = I.first + (valid ? (uint32_t)gl : I.count - 1u);
  const size_t e = nd.elem0 + idx;
  const bool write = valid && !P.dry;

  // Gamma2(z_i), Gamma2(-v_i)
  const double zi = P.z[e], vi = P.v[e];
  const uint64_t qz = quant(zi, P.zmin, P.scale, P.qmax, P.status);
  const uint64_t qv = quant(-vi, P.zmin, P.scale, P.qmax, P.status);

  // z-hat, (-v)-hat: r from stream (t << 8) | kind, counter e (the global index)
#pragma unroll 1
  for (int which = 0; which < 2; ++which) {
    const uint32_t sid = (round << 8) | (which ? 2u : 1u);
    gen_r(X, P.seed, sid, e, Lh + 2, L2);
    gm_u64(GM, A, which ? qv : qz, K.enc.nwords, Lh, L2);
    enc_half_f<Lh, T, MS>(K.enc.mp, bmod<Lh, 0>(), K.enc.ep, K.enc.lp, bprime<Lh, 0>(), X, GM, CP, A, B, C, TT, tab, bsh,
                      g);
    enc_half_f<Lh, T, MS>(K.enc.mq, bmod<Lh, 1>(), K.enc.eq, K.enc.lq, bprime<Lh, 1>(), X, GM, CQ, A, B, C, TT, tab, bsh,
                      g);
    // Eq. (gA-C-B): c = c_p + [(c_q - c_p) (p^2)^-1 mod q^2] p^2
    if (g_sub(A, CQ, CP, Lh)) g_add(A, A, PArr{K.enc.mq.n}, Lh);
    grp_mont<Lh, T, MS>(C, A, const_col(K.enc.pinv2R), K.enc.mq.n, K.enc.mq.np, TT, g);
    g_mul(X, C, Lh, PArr{K.enc.p2}, Lh);
    const Col OUT = which ? CV : CZ;
    uint64_t c = 0;
    for (int j = 0; j < L2; ++j) {
      c += (uint64_t)X[j] + (j < Lh ? CP[j] : 0u);
      OUT[j] = (uint32_t)c;
      c >>= 32;
    }
    if (write) write_tiled<T>((which ? P.vhat : P.zhat) + nd.ct_off, idx, OUT, L2, g);
    __syncwarp();
  }

  // s-hat R = (z-hat (-v)-hat R^-1) R^3 R^-1 mod n^2
  grp_mont<L2, T, MS>(C, CZ, CV, K.n2.n, K.n2.np, TT, g);
  grp_mont<L2, T, MS>(A, C, const_col(K.n2.r3), K.n2.n, K.n2.np, TT, g);
  // (s-hat^b) R, digits of the widest b of the warp
  const uint64_t bi = P.b[e];
  const uint32_t hi = __reduce_or_sync(PC2_FULL, (uint32_t)(bi >> 32));
  const uint32_t lo = __reduce_or_sync(PC2_FULL, (uint32_t)bi);
  const int bits = hi ? 64 - __clz(hi) : (lo ? 32 - __clz(lo) : 1);
  grp_pow_u64<L2, T, MS>(C, A, bi, kScalWin, (bits + kScalWin - 1) / kScalWin, tab, K.n2.r1, K.n2.n, K.n2.np, TT, g);
  // x-hat = alpha-hat * s-hat^b mod n^2
  for (int j = 0; j < L2; ++j) B[j] = P.alpha_hat[nd.ct_off + tiled_index(idx, j, L2)];
  grp_mont<L2, T, MS>(X, C, B, K.n2.n, K.n2.np, TT, g);
  if (write) write_tiled<T>(P.xhat + nd.ct_off, idx, X, L2, g);
  __syncwarp();

  // D = decrypt(x-hat): CRT halves, Garner m = m_p + p [(m_q - m_p) p^-1 mod q]
  dec_half_f<Lh, T, MS>(K.dec.mp, bmod<Lh, 0>(), K.dec.ep, K.dec.p, K.dec.pnp, K.dec.pinvlo, K.dec.hpR, X, CP, A, B, C, TT, tab, bsh,
                       g);
  dec_half_f<Lh, T, MS>(K.dec.mq, bmod<Lh, 1>(), K.dec.eq, K.dec.q, K.dec.qnp, K.dec.qinvlo, K.dec.hqR, X, CQ, A, B, C, TT, tab, bsh,
                       g);
  if (g_sub(A, CQ, CP, Lp)) g_add(A, A, PArr{K.dec.q}, Lp);
  grp_mont<Lp, T, MS>(C, A, const_col(K.dec.pinvqR), K.dec.q, K.dec.qnp, TT, g);
  g_mul(X, C, Lp, PArr{K.dec.p}, Lp);
  {
    uint64_t c = 0;
    for (int j = 0; j < Lh; ++j) {
      c += (uint64_t)X[j] + (j < Lp ? CP[j] : 0u);
      X[j] = (uint32_t)c;
      c >>= 32;
    }
  }

  // exact decode with N_k = 1: X = D + mS S + 2 mS b + mS (a_z + a_v) + 2 mS^2
  uint32_t top = 0;
  for (int j = 4; j < Lh; ++j) top |= X[j];
  const unsigned __int128 d = (unsigned __int128)X[0] | ((unsigned __int128)X[1] << 32) |
                              ((unsigned __int128)X[2] << 64) | ((unsigned __int128)X[3] << 96);
  __int128 Xv = (__int128)d;
  Xv += (__int128)P.mS * P.S;
  Xv += (__int128)2 * P.mS * (__int128)bi;
  Xv += (__int128)P.mS * (__int128)(qz + qv);
  Xv += (__int128)2 * P.mS * P.mS;
  const bool bad = top != 0u || Xv > (__int128)0x7fffffffffffffffLL || Xv < -(__int128)0x7fffffffffffffffLL;
  if (valid && bad) atomicOr(P.status, PC2_ST_RANGE);
  const double xi = __dmul_rn(__ll2double_rn((long long)Xv), P.inv_s2);
  double zn = zi, vn = vi;
  zv_update(xi, zn, vn, P.kappa);
  if (write && g.k == 0) {
    P.x[e] = xi;
    P.z[e] = zn;
    P.v[e] = vn;
  }
  __syncwarp();
}

__global__ void __launch_bounds__(kThreads, 3) k_batch_round(const __grid_constant__ BatchParams P) {
  extern __shared__ uint32_t bsh_all[];
  __shared__ uint32_t s_item;
  const uint32_t round = *(volatile const uint32_t*)&P.ctl->round;
  uint32_t* cta = P.scratch + (size_t)blockIdx.x * P.cta_words;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(&P.ctl->next, 1u);
    __syncthreads();
    const uint32_t it = s_item;
    __syncthreads();
    if (it >= P.nitems) break;
    const BatchItem I = P.items[it];
    switch (I.cls) {
      case 0: batch_item<8, batch_lanes(8)>(P, I, round, cta, bsh_all); break;
      case 1: batch_item<16, batch_lanes(16)>(P, I, round, cta, bsh_all); break;
      case 2: batch_item<32, batch_lanes(32)>(P, I, round, cta, bsh_all); break;
      case 3: batch_item<64, batch_lanes(64)>(P, I, round, cta, bsh_all); break;
      case 4: batch_item<96, batch_lanes(96)>(P, I, round, cta, bsh_all); break;
      default: break;
    }
  }
  // the last CTA re-arms the work list and advances the round
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&P.ctl->done, 1u) == gridDim.x - 1u) {
      P.ctl->next = 0u;
      P.ctl->done = 0u;
      if (!P.dry) P.ctl->round = round + 1u;
      __threadfence();
    }
  }
}

// Plain per-node path: decode (N_k = 1) and z/v update of n elements of one
// node; D tiled with Lh limbs, node-local indices.
__global__ void k_batch_update(const uint32_t* __restrict__ D, int Lh, size_t n, const uint64_t* __restrict__ zq,
                               const uint64_t* __restrict__ vq, const uint64_t* __restrict__ b, long long mS,
                               long long S, double inv_s2, double kappa, double* __restrict__ x,
                               double* __restrict__ z, double* __restrict__ v, int* status, uint32_t* round_ctr) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    uint32_t top = 0;
    for (int j = 4; j < Lh; ++j) top |= D[tiled_index(i, j, Lh)];
    const unsigned __int128 d = (unsigned __int128)D[tiled_index(i, 0, Lh)] |
                                ((unsigned __int128)D[tiled_index(i, 1, Lh)] << 32) |
                                ((unsigned __int128)D[tiled_index(i, 2, Lh)] << 64) |
                                ((unsigned __int128)D[tiled_index(i, 3, Lh)] << 96);
    __int128 Xv = (__int128)d;
    Xv += (__int128)mS * S;
    Xv += (__int128)2 * mS * (__int128)b[i];
    Xv += (__int128)mS * (__int128)(zq[i] + vq[i]);
    Xv += (__int128)2 * mS * mS;
    if (top != 0u || Xv > (__int128)0x7fffffffffffffffLL || Xv < -(__int128)0x7fffffffffffffffLL)
      atomicOr(status, PC2_ST_RANGE);
    const double xi = __dmul_rn(__ll2double_rn((long long)Xv), inv_s2);
    double zi = z[i], vi = v[i];
    zv_update(xi, zi, vi, kappa);
    x[i] = xi;
    z[i] = zi;
    v[i] = vi;
  }
  if (round_ctr && blockIdx.x == 0 && threadIdx.x == 0) *round_ctr += 1u;
}

int batch_blocks_per_sm(size_t smem) {
  int per = 0;
  if (cudaFuncSetAttribute(k_batch_round, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_round, kThreads, smem) != cudaSuccess) return -1;
  return per;
}

int launch_batch_round(const BatchParams& P, const BatchConstMods* d_mods, size_t smem, int grid, cudaStream_t st) {
  if (cudaMemcpyToSymbolAsync(c_bmods, d_mods, sizeof(BatchConstMods), 0, cudaMemcpyDeviceToDevice, st) !=
      cudaSuccess)
    return PC2_ECUDA;
  k_batch_round<<<grid, kThreads, smem, st>>>(P);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

int launch_batch_update(const uint32_t* D, int Lh, size_t n, const uint64_t* zq, const uint64_t* vq,
                        const uint64_t* b, long long mS, long long S, double inv_s2, double kappa, double* x,
                        double* z, double* v, int* status, uint32_t* round_ctr, int sms, cudaStream_t st) {
  size_t blocks = (n + 255) / 256;
  if (blocks > (size_t)sms * 8) blocks = (size_t)sms * 8;
  if (blocks < 1) blocks = 1;
  k_batch_update<<<(unsigned)blocks, 256, 0, st>>>(D, Lh, n, zq, vq, b, mS, S, inv_s2, kappa, x, z, v, status,
                                                    round_ctr);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

}  // namespace pc2
