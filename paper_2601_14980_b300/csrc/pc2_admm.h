// pc2_admm.h -- internal declarations of the ADMM-side launchers.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "pc2_params.h"

namespace pc2 {

int launch_quantize(const double* u, size_t n, double zmin, double scale, double qmax, int negate, uint64_t* q,
                    int* status, uint32_t* bitlen_or, int sms, cudaStream_t st);
int launch_dequantize(const uint64_t* q, size_t n, double zmin, double inv_scale, double* u, int sms, cudaStream_t st);
int launch_decode_matvec(const uint32_t* D, int Lh, size_t n, const long long* brow, const unsigned long long* asum,
                         const int* nk, long long mS, long long S, double inv_s2, double* x, int* status, int sms,
                         cudaStream_t st);
int launch_admm_quant(const double* z, const double* v, int N, const int* node_of, double zmin, double scale,
                      double qmax, uint64_t* zq, uint64_t* vq, unsigned long long* asum, int* status, int sms,
                      cudaStream_t st);
int launch_admm_update(const uint32_t* D, int Lh, int N, const int* node_of, const int* node_size,
                       const long long* brow, const unsigned long long* asum, long long mS, long long S, double inv_s2,
                       double kappa, double* x, double* z, double* v, int* status, uint32_t* round_ctr, int sms,
                       cudaStream_t st);
int launch_narrow(const uint64_t* q, size_t n, uint32_t* out, int* status, int sms, cudaStream_t st);
int launch_rowsum(const uint32_t* bq, const long long* boff, const int* node_of, const int* node_off, int N,
                  long long* brow, int sms, cudaStream_t st);
int launch_zv_update(const double* x, double* z, double* v, int N, double kappa, int sms, cudaStream_t st);
int launch_dis_xupdate(const double* alpha, const double* Bbar, const long long* boff, const int* node_of,
                       const int* node_off, const double* z, const double* v, double* x, int N, int sms,
                       cudaStream_t st);
template <int L2, int T>
int launch_to_mont_rows(const ModConst<L2>& M, const uint32_t* s, int N, uint32_t* smont, int sms, cudaStream_t st);
template <int L2, int T>
size_t matvec_scratch_words(int c, int grid);
template <int L2, int T>
int launch_matvec(const MatvecParams<L2>& P, const uint32_t* alpha_hat, const uint32_t* smont, const uint32_t* bq,
                  const long long* boff, const int* node_off, const int* tile_node, const int* tile_row0,
                  uint32_t* out, uint32_t* scratch, int grid, cudaStream_t st);
template <int L2, int T>
int matvec_grid(int ntiles, int sms);
// Window-parallel form of the same product (few row tiles): part holds
// nwin x N partial products (tiled, L2 limbs).
template <int L2, int T>
int launch_matvec_win(const MatvecParams<L2>& P, const uint32_t* alpha_hat, const uint32_t* smont, const uint32_t* bq,
                      const long long* boff, const int* node_off, const int* tile_node, const int* tile_row0, int N,
                      uint32_t* part, uint32_t* out, uint32_t* scratch, int grid, int sms, cudaStream_t st);
template <int L2, int T>
int matvec_win_grid(int items, int sms);


}  // namespace pc2
