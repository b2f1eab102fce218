// admm_kernels.cuh -- templated kernels of the encrypted matvec (Montgomery
// form of s-hat and the bucket-method matvec) and their launchers; the
// inst_mv_*.cu files instantiate them per operand size and lane count.
#pragma once
#include <cuda_runtime.h>

#include "mont.cuh"
#include "pc2_admm.h"
#include "pc2_kernels.h"

namespace pc2 {

// ------------------------------------------------------------------ Montgomery form of s-hat
// smont[j * L2 + w] = word w of s_j * R mod n^2 (row-major: a CTA stages a row with one coalesced read).
template <int L2, int T>
__global__ void __launch_bounds__(kThreads) k_to_mont_rows(const __grid_constant__ ModConst<L2> M,
                                                           const uint32_t* __restrict__ s, int N,
                                                           uint32_t* __restrict__ smont) {
  constexpr int S = L2 / T;
  extern __shared__ uint32_t bsh_all[];
  const Grp<T> g;
  const int G = blockDim.x / T, gl = threadIdx.x / T;
  const Col bsh{bsh_all + gl, G};
  RegN<S> rn;
  if constexpr (T > 1) rn = reg_n<S, T>(M.n, g);
  for (int base = blockIdx.x * G; base < N; base += gridDim.x * G) {
    int e = base + gl;
    const bool valid = e < N;
    if (!valid) e = N - 1;
    uint32_t a[S];
#pragma unroll
    for (int j = 0; j < S; ++j) a[j] = s[tiled_index((size_t)e, g.k * S + j, L2)];
#pragma unroll
    for (int j = 0; j < S; ++j) bsh[g.k * S + j] = M.r2[g.k * S + j];
    __syncwarp();
    if constexpr (T == 1) mont_mul<S, T>(a, bsh.p, bsh.s, ParamN{M.n}, M.np, g);
    else mont_mul<S, T>(a, bsh.p, bsh.s, rn, M.np, g);
    __syncwarp();
    if (valid) {
#pragma unroll
      for (int j = 0; j < S; ++j) smont[(size_t)e * L2 + g.k * S + j] = a[j];
    }
  }
}

// ------------------------------------------------------------------ encrypted matvec
template <int L2, int T>
__global__ void __launch_bounds__(kThreads, 2) k_matvec(const __grid_constant__ MatvecParams<L2> P,
                                                      const uint32_t* __restrict__ alpha_hat,
                                                      const uint32_t* __restrict__ smont,
                                                      const uint32_t* __restrict__ bq,
                                                      const long long* __restrict__ boff,
                                                      const int* __restrict__ node_off,
                                                      const int* __restrict__ tile_node,
                                                      const int* __restrict__ tile_row0,
                                                      uint32_t* __restrict__ out, uint32_t* __restrict__ scratch) {
  constexpr int S = L2 / T;
  extern __shared__ uint32_t sh[];
  const Grp<T> g;
  const int G = blockDim.x / T, gl = threadIdx.x / T;
  const int Gtot = gridDim.x * G, gg = blockIdx.x * G + gl;
  uint32_t* sj = sh;                       // the shared base s_j (L2 words, read by every group)
  const Col bsh{sh + L2 + gl, G};          // per-group operand column
  const int nb = 1 << P.c;
  auto col = [&](int w) { return Col{scratch + (size_t)w * Gtot + gg, Gtot}; };
  const Col BK = col(0);                   // buckets: nb x L2 words
  const Col ACC = col(nb * L2), RR = col((nb + 1) * L2), SS = col((nb + 2) * L2);
  RegN<S> rn;
  if constexpr (T > 1) rn = reg_n<S, T>(P.m.n, g);
  auto mm = [&](uint32_t(&a)[S], const uint32_t* b, int bs) {
    if constexpr (T == 1) mont_mul<S, T>(a, b, bs, ParamN{P.m.n}, P.m.np, g);
    else mont_mul<S, T>(a, b, bs, rn, P.m.np, g);
  };
  const uint32_t dmask = (uint32_t)nb - 1u;
  for (int tile = blockIdx.x; tile < P.ntiles; tile += gridDim.x) {
    const int k = tile_node[tile];
    const int o = node_off[k], nk = node_off[k + 1] - o;
    int i = tile_row0[tile] + gl;  // global row
    const bool valid = i < o + nk;
    if (!valid) i = o + nk - 1;
    const uint32_t* brow = bq + boff[k] + (long long)(i - o) * nk;
    uint32_t a[S];
    for (int win = P.nwin - 1; win >= 0; --win) {
      // acc <- acc^(2^c)
      if (win == P.nwin - 1) {
#pragma unroll
        for (int j = 0; j < S; ++j) a[j] = P.m.r1[g.k * S + j];
      } else {
        load_seg(a, ACC, g);
        for (int q = 0; q < P.c; ++q) {
          store_seg(bsh, a, g);
          __syncwarp();
          mm(a, bsh.p, bsh.s);
          __syncwarp();
        }
      }
      store_seg(ACC, a, g);
      // buckets <- 1
      for (int d = 0; d < nb; ++d)
#pragma unroll
        for (int j = 0; j < S; ++j) BK[d * L2 + g.k * S + j] = P.m.r1[g.k * S + j];
      for (int jj = 0; jj < nk; ++jj) {
        __syncthreads();
        for (int w = threadIdx.x; w < L2; w += blockDim.x) sj[w] = smont[(size_t)(o + jj) * L2 + w];
        __syncthreads();
        const int d = (int)((brow[jj] >> (win * P.c)) & dmask);
        const Col B = BK.off(d * L2);
        load_seg(a, B, g);
        mm(a, sj, 1);
        store_seg(B, a, g);
      }
      // S = prod_d bucket_d^d via R_d = prod_{e >= d} bucket_e, S = prod_d R_d
      load_seg(a, BK.off((nb - 1) * L2), g);
      store_seg(RR, a, g);
      store_seg(SS, a, g);
      for (int d = nb - 2; d >= 1; --d) {
        __syncwarp();
        load_seg(a, RR, g);
        {
          uint32_t t[S];
          load_seg(t, BK.off(d * L2), g);
          store_seg(bsh, t, g);
        }
        __syncwarp();
        mm(a, bsh.p, bsh.s);  // R <- R * bucket_d
        __syncwarp();
        store_seg(RR, a, g);
        store_seg(bsh, a, g);
        __syncwarp();
        load_seg(a, SS, g);
        mm(a, bsh.p, bsh.s);  // S <- S * R
        __syncwarp();
        store_seg(SS, a, g);
      }
      // acc <- acc * S
      __syncwarp();
      load_seg(a, SS, g);
      store_seg(bsh, a, g);
      __syncwarp();
      load_seg(a, ACC, g);
      mm(a, bsh.p, bsh.s);
      __syncwarp();
      store_seg(ACC, a, g);
    }
    // x-hat_i = alpha-hat_i (+) result: mont(acc, alpha-hat_i) with alpha-hat plain
#pragma unroll
    for (int j = 0; j < S; ++j) bsh[g.k * S + j] = alpha_hat[tiled_index((size_t)i, g.k * S + j, L2)];
    __syncwarp();
    mm(a, bsh.p, bsh.s);
    __syncwarp();
    if (valid) {
#pragma unroll
      for (int j = 0; j < S; ++j) out[tiled_index((size_t)i, g.k * S + j, L2)] = a[j];
    }
  }
}

template <int L2, int T>
int launch_to_mont_rows(const ModConst<L2>& M, const uint32_t* s, int N, uint32_t* smont, int sms, cudaStream_t st) {
  const size_t smem = (size_t)L2 * (kThreads / T) * 4;
  auto kern = k_to_mont_rows<L2, T>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return PC2_ECUDA;
  int grid = (N + (kThreads / T) - 1) / (kThreads / T);
  if (grid > sms * 4) grid = sms * 4;
  kern<<<grid, kThreads, smem, st>>>(M, s, N, smont);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

// ------------------------------------------------------------------ window-parallel matvec
// The same x-hat as k_matvec with the bucket windows of a row computed by
// different CTAs (k_matvec_win: one (row tile, window) pair per work item,
// writing the window's product prod_d bucket_d^d to `part`), then combined
// per row by Horner's rule (k_matvec_join: acc <- acc^(2^c) * part_win from
// the top window down, then alpha-hat).  For problems with few row tiles,
// where k_matvec would leave most SMs idle.  part: element (win * N + i) of a
// tiled array of L2-limb numbers (N = rows of all nodes).
template <int L2, int T>
__global__ void __launch_bounds__(kThreads, 2) k_matvec_win(const __grid_constant__ MatvecParams<L2> P,
                                                          const uint32_t* __restrict__ smont,
                                                          const uint32_t* __restrict__ bq,
                                                          const long long* __restrict__ boff,
                                                          const int* __restrict__ node_off,
                                                          const int* __restrict__ tile_node,
                                                          const int* __restrict__ tile_row0, int N,
                                                          uint32_t* __restrict__ part, uint32_t* __restrict__ scratch) {
  constexpr int S = L2 / T;
  extern __shared__ uint32_t sh[];
  const Grp<T> g;
  const int G = blockDim.x / T, gl = threadIdx.x / T;
  const int Gtot = gridDim.x * G, gg = blockIdx.x * G + gl;
  uint32_t* sj = sh;
  const Col bsh{sh + L2 + gl, G};
  const int nb = 1 << P.c;
  auto col = [&](int w) { return Col{scratch + (size_t)w * Gtot + gg, Gtot}; };
  const Col BK = col(0), RR = col((nb + 1) * L2), SS = col((nb + 2) * L2);
  RegN<S> rn;
  if constexpr (T > 1) rn = reg_n<S, T>(P.m.n, g);
  auto mm = [&](uint32_t(&a)[S], const uint32_t* b, int bs) {
    if constexpr (T == 1) mont_mul<S, T>(a, b, bs, ParamN{P.m.n}, P.m.np, g);
    else mont_mul<S, T>(a, b, bs, rn, P.m.np, g);
  };
  const uint32_t dmask = (uint32_t)nb - 1u;
  const int items = P.ntiles * P.nwin;
  for (int it = blockIdx.x; it < items; it += gridDim.x) {
    const int tile = it / P.nwin, win = it % P.nwin;
    const int k = tile_node[tile];
    const int o = node_off[k], nk = node_off[k + 1] - o;
    int i = tile_row0[tile] + gl;
    const bool valid = i < o + nk;
    if (!valid) i = o + nk - 1;
    const uint32_t* brow = bq + boff[k] + (long long)(i - o) * nk;
    uint32_t a[S];
    for (int d = 0; d < nb; ++d)
#pragma unroll
      for (int j = 0; j < S; ++j) BK[d * L2 + g.k * S + j] = P.m.r1[g.k * S + j];
    for (int jj = 0; jj < nk; ++jj) {
      __syncthreads();
      for (int w = threadIdx.x; w < L2; w += blockDim.x) sj[w] = smont[(size_t)(o + jj) * L2 + w];
      __syncthreads();
      const int d = (int)((brow[jj] >> (win * P.c)) & dmask);
      const Col B = BK.off(d * L2);
      load_seg(a, B, g);
      mm(a, sj, 1);
      store_seg(B, a, g);
    }
    // prod_d bucket_d^d = prod_d R_d with R_d = prod_{e >= d} bucket_e
    load_seg(a, BK.off((nb - 1) * L2), g);
    store_seg(RR, a, g);
    store_seg(SS, a, g);
    for (int d = nb - 2; d >= 1; --d) {
      __syncwarp();
      load_seg(a, RR, g);
      {
        uint32_t t[S];
        load_seg(t, BK.off(d * L2), g);
        store_seg(bsh, t, g);
      }
      __syncwarp();
      mm(a, bsh.p, bsh.s);
      __syncwarp();
      store_seg(RR, a, g);
      store_seg(bsh, a, g);
      __syncwarp();
      load_seg(a, SS, g);
      mm(a, bsh.p, bsh.s);
      __syncwarp();
      store_seg(SS, a, g);
    }
    __syncwarp();
    load_seg(a, SS, g);
    if (valid) {
#pragma unroll
      for (int j = 0; j < S; ++j) part[tiled_index((size_t)win * N + i, g.k * S + j, L2)] = a[j];
    }
    __syncwarp();
  }
}

template <int L2, int T>
__global__ void __launch_bounds__(kThreads, 2) k_matvec_join(const __grid_constant__ MatvecParams<L2> P,
                                                           const uint32_t* __restrict__ alpha_hat,
                                                           const uint32_t* __restrict__ part, int N,
                                                           uint32_t* __restrict__ out) {
  constexpr int S = L2 / T;
  extern __shared__ uint32_t sh[];
  const Grp<T> g;
  const int G = blockDim.x / T, gl = threadIdx.x / T;
  const Col bsh{sh + gl, G};
  RegN<S> rn;
  if constexpr (T > 1) rn = reg_n<S, T>(P.m.n, g);
  auto mm = [&](uint32_t(&a)[S], const uint32_t* b, int bs) {
    if constexpr (T == 1) mont_mul<S, T>(a, b, bs, ParamN{P.m.n}, P.m.np, g);
    else mont_mul<S, T>(a, b, bs, rn, P.m.np, g);
  };
  for (int base = blockIdx.x * G; base < N; base += gridDim.x * G) {
    int i = base + gl;
    const bool valid = i < N;
    if (!valid) i = N - 1;
    uint32_t a[S];
#pragma unroll
    for (int j = 0; j < S; ++j) a[j] = part[tiled_index((size_t)(P.nwin - 1) * N + i, g.k * S + j, L2)];
    for (int win = P.nwin - 2; win >= 0; --win) {
      for (int q = 0; q < P.c; ++q) {
        store_seg(bsh, a, g);
        __syncwarp();
        mm(a, bsh.p, bsh.s);
        __syncwarp();
      }
#pragma unroll
      for (int j = 0; j < S; ++j) bsh[g.k * S + j] = part[tiled_index((size_t)win * N + i, g.k * S + j, L2)];
      __syncwarp();
      mm(a, bsh.p, bsh.s);
      __syncwarp();
    }
#pragma unroll
    for (int j = 0; j < S; ++j) bsh[g.k * S + j] = alpha_hat[tiled_index((size_t)i, g.k * S + j, L2)];
    __syncwarp();
    mm(a, bsh.p, bsh.s);
    __syncwarp();
    if (valid) {
#pragma unroll
      for (int j = 0; j < S; ++j) out[tiled_index((size_t)i, g.k * S + j, L2)] = a[j];
    }
  }
}

template <int L2, int T>
int launch_matvec_win(const MatvecParams<L2>& P, const uint32_t* alpha_hat, const uint32_t* smont, const uint32_t* bq,
                      const long long* boff, const int* node_off, const int* tile_node, const int* tile_row0, int N,
                      uint32_t* part, uint32_t* out, uint32_t* scratch, int grid, int sms, cudaStream_t st) {
  const size_t smem1 = (size_t)L2 * (kThreads / T + 1) * 4, smem2 = (size_t)L2 * (kThreads / T) * 4;
  auto k1 = k_matvec_win<L2, T>;
  auto k2 = k_matvec_join<L2, T>;
  if (cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1) != cudaSuccess ||
      cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2) != cudaSuccess)
    return PC2_ECUDA;
  k1<<<grid, kThreads, smem1, st>>>(P, smont, bq, boff, node_off, tile_node, tile_row0, N, part, scratch);
  if (cudaGetLastError() != cudaSuccess) return PC2_ECUDA;
  const int G = kThreads / T;
  int g2 = (N + G - 1) / G;
  if (g2 > 2 * sms) g2 = 2 * sms;
  k2<<<g2, kThreads, smem2, st>>>(P, alpha_hat, part, N, out);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

// CTAs of k_matvec_win that can be resident (the grid the window-parallel
// launch uses; its scratch is matvec_scratch_words(c, grid)).
template <int L2, int T>
int matvec_win_grid(int items, int sms) {
  int per = 0;
  const size_t smem = (size_t)L2 * (kThreads / T + 1) * 4;
  auto kern = k_matvec_win<L2, T>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kThreads, smem) != cudaSuccess || per < 1) return -1;
  const int g = per * sms;
  return items < g ? items : g;
}

template <int L2, int T>
size_t matvec_scratch_words(int c, int grid) {
  return (size_t)((1 << c) + 3) * L2 * (size_t)grid * (kThreads / T);
}

template <int L2, int T>
int launch_matvec(const MatvecParams<L2>& P, const uint32_t* alpha_hat, const uint32_t* smont, const uint32_t* bq,
                  const long long* boff, const int* node_off, const int* tile_node, const int* tile_row0,
                  uint32_t* out, uint32_t* scratch, int grid, cudaStream_t st) {
  const size_t smem = (size_t)L2 * (kThreads / T + 1) * 4;
  auto kern = k_matvec<L2, T>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return PC2_ECUDA;
  kern<<<grid, kThreads, smem, st>>>(P, alpha_hat, smont, bq, boff, node_off, tile_node, tile_row0, out, scratch);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

template <int L2, int T>
int matvec_grid(int ntiles, int sms) {
  int per = 0;
  const size_t smem = (size_t)L2 * (kThreads / T + 1) * 4;
  auto kern = k_matvec<L2, T>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kThreads, smem) != cudaSuccess || per < 1) return -1;
  const int g = per * sms;
  return ntiles < g ? ntiles : g;
}

}  // namespace pc2
