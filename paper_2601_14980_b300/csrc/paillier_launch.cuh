#pragma once
#include "paillier_kernels.cuh"

namespace pc2 {

template <class K>
inline int occupancy_grid(K kern, size_t smem, int sms) {
  int per = 0;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kThreads, smem) != cudaSuccess) return -1;
  if (per < 1) return -1;
  return per * sms;
}

template <int Lh, int T>
int launch_enc_crt(const EncCrtParams<Lh>& P, const uint64_t* m64, const uint32_t* mwide, size_t count, uint32_t* out,
                   ScratchFn scratch_fn, void* sctx, int* status, int sms, cudaStream_t st, size_t base) {
  const size_t smem = (size_t)Lh * (kThreads / T) * 4;
  auto kern = k_enc_crt<Lh, T>;
  const int grid = occupancy_grid(kern, smem, sms);
  if (grid < 0) return PC2_ECUDA;
  const int w = P.ep.w > P.eq.w ? P.ep.w : P.eq.w;
  const int tabw = (1 << (w - 1)) * Lh;
  const size_t per_group = (size_t)tabw + 8 * (size_t)(2 * Lh + 4);
  uint32_t* scratch = scratch_fn(sctx, per_group * (size_t)grid * (kThreads / T) * 4);
  if (!scratch) return PC2_ENOMEM;
  kern<<<grid, kThreads, smem, st>>>(P, m64, mwide, count, out, scratch, tabw, status, base);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

template <int L2, int T>
int launch_enc_pub(const EncPubParams<L2>& P, const uint64_t* m64, const uint32_t* mwide, size_t count, uint32_t* out,
                   ScratchFn scratch_fn, void* sctx, int* status, int sms, cudaStream_t st) {
  const size_t smem = (size_t)L2 * (kThreads / T) * 4;
  auto kern = k_enc_pub<L2, T>;
  const int grid = occupancy_grid(kern, smem, sms);
  if (grid < 0) return PC2_ECUDA;
  const int tabw = (1 << (P.e.w - 1)) * L2;
  const size_t per_group = (size_t)tabw + 4 * (size_t)(L2 + 4);
  uint32_t* scratch = scratch_fn(sctx, per_group * (size_t)grid * (kThreads / T) * 4);
  if (!scratch) return PC2_ENOMEM;
  kern<<<grid, kThreads, smem, st>>>(P, m64, mwide, count, out, scratch, tabw, status);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

template <int Lh, int T>
int launch_dec_crt(const DecParams<Lh>& P, const uint32_t* ct, size_t count, uint32_t* out, ScratchFn scratch_fn,
                   void* sctx, int sms, cudaStream_t st, size_t base) {
  const size_t smem = (size_t)Lh * (kThreads / T) * 4;
  auto kern = k_dec_crt<Lh, T>;
  const int grid = occupancy_grid(kern, smem, sms);
  if (grid < 0) return PC2_ECUDA;
  const int w = P.ep.w > P.eq.w ? P.ep.w : P.eq.w;
  const int tabw = (1 << (w - 1)) * Lh;
  const size_t per_group = (size_t)tabw + 7 * (size_t)(2 * Lh + 4);
  uint32_t* scratch = scratch_fn(sctx, per_group * (size_t)grid * (kThreads / T) * 4);
  if (!scratch) return PC2_ENOMEM;
  kern<<<grid, kThreads, smem, st>>>(P, ct, count, out, scratch, tabw, base);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

// Decryption into a fixed scratch region of `scratch_words` words: the
// persistent grid is cut down to the CTAs whose scratch fits.
template <int Lh, int T>
int launch_dec_crt_fixed(const DecParams<Lh>& P, const uint32_t* ct, size_t count, uint32_t* out, uint32_t* scratch,
                         size_t scratch_words, int sms, cudaStream_t st) {
  const size_t smem = (size_t)Lh * (kThreads / T) * 4;
  auto kern = k_dec_crt<Lh, T>;
  int grid = occupancy_grid(kern, smem, sms);
  if (grid < 0) return PC2_ECUDA;
  const int w = P.ep.w > P.eq.w ? P.ep.w : P.eq.w;
  const int tabw = (1 << (w - 1)) * Lh;
  const size_t per_cta = ((size_t)tabw + 7 * (size_t)(2 * Lh + 4)) * (kThreads / T);
  if (per_cta > scratch_words) return PC2_ERANGE;
  const size_t fit = scratch_words / per_cta;
  if ((size_t)grid > fit) grid = (int)fit;
  kern<<<grid, kThreads, smem, st>>>(P, ct, count, out, scratch, tabw, (size_t)0);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

template <int L2, int T>
int launch_hom_sum(const HomParams<L2>& P, size_t count, uint32_t* out, int sms, cudaStream_t st, size_t base) {
  const size_t smem = (size_t)L2 * (kThreads / T) * 4;
  auto kern = k_hom_sum<L2, T>;
  int grid = occupancy_grid(kern, smem, sms);
  if (grid < 0) return PC2_ECUDA;
  const size_t groups_needed = (count + (kThreads / T) - 1) / (kThreads / T);
  if ((size_t)grid > groups_needed) grid = (int)groups_needed;
  kern<<<grid, kThreads, smem, st>>>(P, count, out, base);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

template <int L2, int T>
int launch_hom_scal(const HomParams<L2>& P, const uint32_t* ct, const uint64_t* k, size_t count, uint32_t* out,
                    ScratchFn scratch_fn, void* sctx, int sms, cudaStream_t st) {
  const size_t smem = (size_t)L2 * (kThreads / T) * 4;
  auto kern = k_hom_scal<L2, T>;
  const int grid = occupancy_grid(kern, smem, sms);
  if (grid < 0) return PC2_ECUDA;
  const size_t per_group = (size_t)(1 << P.w) * L2;
  uint32_t* scratch = scratch_fn(sctx, per_group * (size_t)grid * (kThreads / T) * 4);
  if (!scratch) return PC2_ENOMEM;
  kern<<<grid, kThreads, smem, st>>>(P, ct, k, count, out, scratch);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

template <int L2, int T>
int launch_hom_scal_wide(const HomParams<L2>& P, const uint32_t* ct, const uint32_t* kw, size_t count, uint32_t* out,
                         ScratchFn scratch_fn, void* sctx, int sms, cudaStream_t st) {
  const size_t smem = (size_t)L2 * (kThreads / T) * 4;
  auto kern = k_hom_scal_wide<L2, T>;
  const int grid = occupancy_grid(kern, smem, sms);
  if (grid < 0) return PC2_ECUDA;
  const size_t per_group = (size_t)(1 << P.w) * L2;
  uint32_t* scratch = scratch_fn(sctx, per_group * (size_t)grid * (kThreads / T) * 4);
  if (!scratch) return PC2_ENOMEM;
  kern<<<grid, kThreads, smem, st>>>(P, ct, kw, count, out, scratch);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

// Split-halves variants (T > 1): same arguments, same results.
template <int Lh, int T>
int launch_enc_crt2(const EncCrtParams<Lh>& P, const uint64_t* m64, const uint32_t* mwide, size_t count, uint32_t* out,
                   ScratchFn scratch_fn, void* sctx, int* status, int sms, cudaStream_t st, size_t base) {
  const size_t smem = (size_t)Lh * (kThreads / T) * 4;
  auto kern = k_enc_crt2<Lh, T>;
  const int grid = occupancy_grid(kern, smem, sms);
  if (grid < 0) return PC2_ECUDA;
  const int w = P.ep.w > P.eq.w ? P.ep.w : P.eq.w;
  const int tabw = (1 << (w - 1)) * Lh;
  const size_t per_group = (size_t)tabw + 8 * (size_t)(2 * Lh + 4);
  uint32_t* scratch = scratch_fn(sctx, per_group * (size_t)grid * (kThreads / T) * 4);
  if (!scratch) return PC2_ENOMEM;
  kern<<<grid, kThreads, smem, st>>>(P, m64, mwide, count, out, scratch, tabw, status, base);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

template <int Lh, int T>
int launch_dec_crt2(const DecParams<Lh>& P, const uint32_t* ct, size_t count, uint32_t* out, ScratchFn scratch_fn,
                   void* sctx, int sms, cudaStream_t st, size_t base) {
  const size_t smem = (size_t)Lh * (kThreads / T) * 4;
  auto kern = k_dec_crt2<Lh, T>;
  const int grid = occupancy_grid(kern, smem, sms);
  if (grid < 0) return PC2_ECUDA;
  const int w = P.ep.w > P.eq.w ? P.ep.w : P.eq.w;
  const int tabw = (1 << (w - 1)) * Lh;
  const size_t per_group = (size_t)tabw + 7 * (size_t)(2 * Lh + 4);
  uint32_t* scratch = scratch_fn(sctx, per_group * (size_t)grid * (kThreads / T) * 4);
  if (!scratch) return PC2_ENOMEM;
  kern<<<grid, kThreads, smem, st>>>(P, ct, count, out, scratch, tabw, base);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

}  // namespace pc2
