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

#include "admm_dev.cuh"
#include "mont.cuh"
#include "pc2_admm.h"
#include "pc2_kernels.h"

namespace pc2 {

// ------------------------------------------------------------------ quantizer
// Memory-bound elementwise kernels (quantize, z/v update): each thread takes
// kUnroll elements one grid stride apart per step and issues all their loads
// before any arithmetic (more bytes in flight per SM than one load per thread).
constexpr int kUnroll = 4;

__global__ void k_quantize(const double* __restrict__ u, size_t n, double zmin, double scale, double qmax, int negate,
                           uint64_t* __restrict__ q, int* status, uint32_t* bitlen_or) {
  uint32_t acc = 0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (kUnroll - 1) * stride < n; i += kUnroll * stride) {
    double x[kUnroll];
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) x[k] = u[i + k * stride];
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      const uint64_t v = quant(negate ? -x[k] : x[k], zmin, scale, qmax, status);
      q[i + k * stride] = v;
      acc |= (uint32_t)(v >> 32) ? 0xffffffffu : (uint32_t)v;
    }
  }
  for (; i < n; i += stride) {
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
  const int stride = gridDim.x * blockDim.x;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (kUnroll - 1) * (long long)stride < N; i += kUnroll * stride) {
    double xs[kUnroll], vs[kUnroll];
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      xs[k] = x[i + k * stride];
      vs[k] = v[i + k * stride];
    }
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      double zi = 0.0, vi = vs[k];
      zv_update(xs[k], zi, vi, kappa);
      z[i + k * stride] = zi;
      v[i + k * stride] = vi;
    }
  }
  for (; i < N; i += stride) {
    double zi = 0.0, vi = v[i];
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

// ------------------------------------------------------------------ inverse quantization
// u = q * (1/S or 1/S^2) + zmin in IEEE double (exact for the quantizer's outputs).
// inv_scale = 2^-k, so q * inv_scale is exact; for q < 2^53 its double is
// assembled from q's bits (integer instructions), above that by the FP64
// conversion and product.  Then one rounded addition of zmin.
__global__ void k_dequantize(const uint64_t* __restrict__ q, size_t n, double zmin, double inv_scale,
                             double* __restrict__ u) {
  // one element per step: unrolled, the compiler predicates the rare FP64
  // branch and runs it for every element (measured slower)
  const int k = 1023 - (int)((__double_as_longlong(inv_scale) >> 52) & 0x7ff);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const uint64_t x = q[i];
    double p;
    if (x == 0u) {
      p = 0.0;
    } else if (x < (1ull << 53)) {
      const int lz = __clzll((long long)x);  // >= 11
      const uint64_t mant = (x << (lz - 11)) & ((1ull << 52) - 1u);
      p = __longlong_as_double(((long long)(1086 - lz - k) << 52) | (long long)mant);
    } else {
      p = __dmul_rn((double)x, inv_scale);
    }
    u[i] = __dadd_rn(p, zmin);
  }
}

// The exact decode of Theorem 1 for one matvec row per thread (no z/v update):
// X = D + mS S + 2 mS brow + mS asum + 2 mS^2 nk, x = fl(X) / S^2.
__global__ void k_decode_matvec(const uint32_t* __restrict__ D, int Lh, size_t n, const long long* __restrict__ brow,
                                const unsigned long long* __restrict__ asum, const int* __restrict__ nk,
                                long long mS, long long S, double inv_s2, double* __restrict__ x, int* status) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    uint32_t hi = 0;
    for (int j = 4; j < Lh; ++j) hi |= D[tiled_index(i, j, Lh)];
    const unsigned __int128 d = (unsigned __int128)D[tiled_index(i, 0, Lh)] |
                                ((unsigned __int128)D[tiled_index(i, 1, Lh)] << 32) |
                                ((unsigned __int128)D[tiled_index(i, 2, Lh)] << 64) |
                                ((unsigned __int128)D[tiled_index(i, 3, Lh)] << 96);
    __int128 X = (__int128)d;
    X += (__int128)mS * S;
    X += (__int128)2 * mS * brow[i];
    X += (__int128)mS * (__int128)asum[i];
    X += (__int128)2 * mS * mS * nk[i];
    if (hi || X > (__int128)0x7fffffffffffffffLL || X < -(__int128)0x7fffffffffffffffLL) atomicOr(status, PC2_ST_RANGE);
    x[i] = __dmul_rn(__ll2double_rn((long long)X), inv_s2);
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

int launch_dequantize(const uint64_t* q, size_t n, double zmin, double inv_scale, double* u, int sms, cudaStream_t st) {
  const int g = grid_for((int)(n < (size_t)1 << 30 ? n : (size_t)1 << 30), 256, sms);
  k_dequantize<<<g, 256, 0, st>>>(q, n, zmin, inv_scale, u);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

int launch_decode_matvec(const uint32_t* D, int Lh, size_t n, const long long* brow, const unsigned long long* asum,
                         const int* nk, long long mS, long long S, double inv_s2, double* x, int* status, int sms,
                         cudaStream_t st) {
  const int g = grid_for((int)(n < (size_t)1 << 30 ? n : (size_t)1 << 30), 256, sms);
  k_decode_matvec<<<g, 256, 0, st>>>(D, Lh, n, brow, asum, nk, mS, S, inv_s2, x, status);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
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

}  // namespace pc2
