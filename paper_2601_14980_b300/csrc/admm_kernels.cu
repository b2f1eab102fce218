// admm_kernels.cu -- the ADMM-side kernels of libpc2.
//
//   k_quantize     Gamma2 / Gamma1 of Eq. (et21) with one public range:
//                  q = rint((u - zmin) S) (Gamma2) or rint((u - zmin) S^2)
//                  (Gamma1), S = 2^log2_scale, IEEE double, no contraction.
//   k_admm_quant   Gamma2(z), Gamma2(-v) of Eq. (uyt12) and the per-node sums
//                  sum_j (Gamma2(z_j) + Gamma2(-v_j)) the exact decode needs.
//   k_matvec       Eq. (itq2) edge side: x-hat_i = alpha-hat_i (+) b (x) s-hat,
//                  i.e. alpha-hat_i * prod_j s-hat_j^{b_ij} mod n^2, per row by
//                  the bucket method: per window of c bits, bucket d collects
//                  the product of the s_j whose digit is d, and
//                  prod_d bucket_d^d comes from two running products.
//   k_admm_update  master side: exact decode of the decrypted integer (Theorem 1
//                  with the matrix product written out), then Eqs. (ty32) and
//                  (u78): z = S_kappa(v + x), v = v + x - z.
//   k_dis_xupdate  plaintext Dis-ADMM local update, Eq. (sldo091):
//                  x_k = alpha_k + Bbar_k (z_k - v_k) (FP64; one warp per row).
//   k_zv_update    Eqs. (ty32), (u78) for the plaintext loop.
#include <cuda_runtime.h>

#include "mont.cuh"
#include "pc2_admm.h"
#include "pc2_kernels.h"

namespace pc2 {

// ------------------------------------------------------------------ quantizer
__device__ __forceinline__ uint64_t quant(double u, double zmin, double scale, double qmax, int* status) {
  const double t = __dmul_rn(__dsub_rn(u, zmin), scale);
  double r = rint(t);
  if (!(r >= 0.0 && r <= qmax)) {  // also catches NaN
    atomicOr(status, PC2_ST_QUANT);
    r = r > qmax ? qmax : 0.0;
  }
  return (uint64_t)r;
}

__global__ void k_quantize(const double* __restrict__ u, size_t n, double zmin, double scale, double qmax, int negate,
                           uint64_t* __restrict__ q, int* status, uint32_t* bitlen_or) {
  uint32_t acc = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double x = negate ? -u[i] : u[i];
    const uint64_t v = quant(x, zmin, scale, qmax, status);
    q[i] = v;
    acc |= (uint32_t)(v >> 32) ? 0xffffffffu : (uint32_t)v;
  }
  if (bitlen_or) {
    acc = __reduce_or_sync(PC2_FULL, acc);
    if ((threadIdx.x & 31) == 0 && acc) atomicOr(bitlen_or, acc);
  }
}

__global__ void k_admm_quant(const double* __restrict__ z, const double* __restrict__ v, int N,
                             const int* __restrict__ node_of, double zmin, double scale, double qmax,
                             uint64_t* __restrict__ zq, uint64_t* __restrict__ vq,
                             unsigned long long* __restrict__ asum, int* status) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const uint64_t a = quant(z[i], zmin, scale, qmax, status);
    const uint64_t b = quant(-v[i], zmin, scale, qmax, status);
    zq[i] = a;
    vq[i] = b;
    atomicAdd(&asum[node_of[i]], (unsigned long long)(a + b));
  }
}

// ------------------------------------------------------------------ exact decode + z/v update
__device__ __forceinline__ void zv_update(double x, double& z, double& v, double kappa) {
  const double a = __dadd_rn(v, x);
  const double zn = a > kappa ? __dsub_rn(a, kappa) : (a < -kappa ? __dadd_rn(a, kappa) : 0.0);
  v = __dsub_rn(a, zn);
  z = zn;
}

// D: decrypted plaintexts, tiled, Lh limbs; the quantized result must fit in
// 128 bits (the upper words are checked to be zero).
__global__ void k_admm_update(const uint32_t* __restrict__ D, int Lh, int N, const int* __restrict__ node_of,
                              const int* __restrict__ node_size, const long long* __restrict__ brow,
                              const unsigned long long* __restrict__ asum, long long mS, long long S,
                              double inv_s2, double kappa, double* __restrict__ x, double* __restrict__ z,
                              double* __restrict__ v, int* status, uint32_t* round_ctr) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    uint32_t hi = 0;
    for (int j = 4; j < Lh; ++j) hi |= D[tiled_index((size_t)i, j, Lh)];
    if (hi) atomicOr(status, PC2_ST_RANGE);
    const unsigned __int128 d = (unsigned __int128)D[tiled_index((size_t)i, 0, Lh)] |
                                ((unsigned __int128)D[tiled_index((size_t)i, 1, Lh)] << 32) |
                                ((unsigned __int128)D[tiled_index((size_t)i, 2, Lh)] << 64) |
                                ((unsigned __int128)D[tiled_index((size_t)i, 3, Lh)] << 96);
    const int k = node_of[i];
    // X = D + mS S + 2 mS sum_j b_ij + mS sum_j a_j + 2 mS^2 N_k   (exact)
    __int128 X = (__int128)d;
    X += (__int128)mS * S;
    X += (__int128)2 * mS * brow[i];
    X += (__int128)mS * (__int128)asum[k];
    X += (__int128)2 * mS * mS * node_size[k];
    if (X > (__int128)0x7fffffffffffffffLL || X < -(__int128)0x7fffffffffffffffLL) atomicOr(status, PC2_ST_RANGE);
    const double xi = __dmul_rn(__ll2double_rn((long long)X), inv_s2);
    double zi = z[i], vi = v[i];
    zv_update(xi, zi, vi, 0.0 + kappa);
    x[i] = xi;
    z[i] = zi;
    v[i] = vi;
  }
  if (round_ctr && blockIdx.x == 0 && threadIdx.x == 0) *round_ctr += 1u;
}

__global__ void k_zv_update(const double* __restrict__ x, double* __restrict__ z, double* __restrict__ v, int N,
                            double kappa) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    double zi = z[i], vi = v[i];
    zv_update(x[i], zi, vi, kappa);
    z[i] = zi;
    v[i] = vi;
  }
}

// One warp per row: x_i = alpha_i + sum_j Bbar_ij (z_j - v_j) over the row's node.
__global__ void k_dis_xupdate(const double* __restrict__ alpha, const double* __restrict__ Bbar,
                              const long long* __restrict__ boff, const int* __restrict__ node_of,
                              const int* __restrict__ node_off, const double* __restrict__ z,
                              const double* __restrict__ v, double* __restrict__ x, int N) {
  const int lane = threadIdx.x & 31;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < N; i += (gridDim.x * blockDim.x) >> 5) {
    const int k = node_of[i];
    const int o = node_off[k], nk = node_off[k + 1] - o;
    const double* row = Bbar + boff[k] + (long long)(i - o) * nk;
    double s = 0.0;
    for (int j = lane; j < nk; j += 32) s = fma(row[j], z[o + j] - v[o + j], s);
#pragma unroll
    for (int off = 16; off; off >>= 1) s += __shfl_down_sync(PC2_FULL, s, off);
    if (lane == 0) x[i] = alpha[i] + s;
  }
}

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

// ------------------------------------------------------------------ set-up helpers
// b_ij as 32-bit digits (Gamma2 values are at most Delta < 2^32).
__global__ void k_narrow(const uint64_t* __restrict__ q, size_t n, uint32_t* __restrict__ out, int* status) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const uint64_t v = q[i];
    if (v >> 32) atomicOr(status, PC2_ST_QUANT);
    out[i] = (uint32_t)v;
  }
}
// brow_i = sum_j b_ij over row i of its node's matrix (one warp per row).
__global__ void k_rowsum(const uint32_t* __restrict__ bq, const long long* __restrict__ boff,
                         const int* __restrict__ node_of, const int* __restrict__ node_off, int N,
                         long long* __restrict__ brow) {
  const int lane = threadIdx.x & 31;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < N; i += (gridDim.x * blockDim.x) >> 5) {
    const int k = node_of[i];
    const int o = node_off[k], nk = node_off[k + 1] - o;
    const uint32_t* row = bq + boff[k] + (long long)(i - o) * nk;
    unsigned long long s = 0;
    for (int j = lane; j < nk; j += 32) s += row[j];
#pragma unroll
    for (int off = 16; off; off >>= 1) s += __shfl_down_sync(PC2_FULL, s, off);
    if (lane == 0) brow[i] = (long long)s;
  }
}

// ------------------------------------------------------------------ launchers
static int grid_for(int n, int threads, int sms) {
  int g = (n + threads - 1) / threads;
  if (g > sms * 8) g = sms * 8;
  return g < 1 ? 1 : g;
}

int launch_quantize(const double* u, size_t n, double zmin, double scale, double qmax, int negate, uint64_t* q,
                    int* status, uint32_t* bitlen_or, int sms, cudaStream_t st) {
  const int g = grid_for((int)(n < (size_t)1 << 30 ? n : (size_t)1 << 30), 256, sms);
  k_quantize<<<g, 256, 0, st>>>(u, n, zmin, scale, qmax, negate, q, status, bitlen_or);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

int launch_admm_quant(const double* z, const double* v, int N, const int* node_of, double zmin, double scale,
                      double qmax, uint64_t* zq, uint64_t* vq, unsigned long long* asum, int* status, int sms,
                      cudaStream_t st) {
  k_admm_quant<<<grid_for(N, 256, sms), 256, 0, st>>>(z, v, N, node_of, zmin, scale, qmax, zq, vq, asum, status);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

int launch_admm_update(const uint32_t* D, int Lh, int N, const int* node_of, const int* node_size,
                       const long long* brow, const unsigned long long* asum, long long mS, long long S, double inv_s2,
                       double kappa, double* x, double* z, double* v, int* status, uint32_t* round_ctr, int sms,
                       cudaStream_t st) {
  k_admm_update<<<grid_for(N, 256, sms), 256, 0, st>>>(D, Lh, N, node_of, node_size, brow, asum, mS, S, inv_s2,
                                                       kappa, x, z, v, status, round_ctr);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

int launch_narrow(const uint64_t* q, size_t n, uint32_t* out, int* status, int sms, cudaStream_t st) {
  k_narrow<<<grid_for((int)(n < (size_t)1 << 30 ? n : (size_t)1 << 30), 256, sms), 256, 0, st>>>(q, n, out, status);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

int launch_rowsum(const uint32_t* bq, const long long* boff, const int* node_of, const int* node_off, int N,
                  long long* brow, int sms, cudaStream_t st) {
  k_rowsum<<<grid_for(N * 32, 256, sms), 256, 0, st>>>(bq, boff, node_of, node_off, N, brow);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

int launch_zv_update(const double* x, double* z, double* v, int N, double kappa, int sms, cudaStream_t st) {
  k_zv_update<<<grid_for(N, 256, sms), 256, 0, st>>>(x, z, v, N, kappa);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

int launch_dis_xupdate(const double* alpha, const double* Bbar, const long long* boff, const int* node_of,
                       const int* node_off, const double* z, const double* v, double* x, int N, int sms,
                       cudaStream_t st) {
  k_dis_xupdate<<<grid_for(N * 32, 256, sms), 256, 0, st>>>(alpha, Bbar, boff, node_of, node_off, z, v, x, N);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
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

#define PC2_ADMM_INST(L2, T)                                                                                       \
  template int launch_to_mont_rows<L2, T>(const ModConst<L2>&, const uint32_t*, int, uint32_t*, int, cudaStream_t); \
  template size_t matvec_scratch_words<L2, T>(int, int);                                                           \
  template int launch_matvec<L2, T>(const MatvecParams<L2>&, const uint32_t*, const uint32_t*, const uint32_t*,    \
                                    const long long*, const int*, const int*, const int*, uint32_t*, uint32_t*,    \
                                    int, cudaStream_t);                                                             \
  template int matvec_grid<L2, T>(int, int);
PC2_ADMM_INST(16, 1)
PC2_ADMM_INST(32, 1)
PC2_ADMM_INST(64, 1)
PC2_ADMM_INST(128, 4)
PC2_ADMM_INST(192, 4)

}  // namespace pc2
