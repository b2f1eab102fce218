// tc_mont.cu -- pc2_mont_sqr: Montgomery squarings of 2048-bit operands with
// the reduction on the tensor cores (engine PC2_ENGINE_TC, the product of
// tc_core.cuh) or on the integer pipe (engine PC2_ENGINE_IMAD, the library's
// CIOS product), the same integers either way.  It isolates the product that
// dominates the fixed-exponent powers of Eq. (itq1) and Sec. III-C.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "../../include/pc2.h"
#include "ctx.hpp"
#include "pc2_kernels.h"
#include "tc_core.cuh"

namespace {

constexpr int kL = 64;
using Core = pc2::tc::Core<kL>;

struct alignas(16) SqrParams {
  pc2::tc::Mod<kL> m;
};

__global__ void __launch_bounds__(pc2::tc::kThreads, 2)
    k_mont_sqr_tc(const __grid_constant__ SqrParams P, const uint32_t* __restrict__ x, size_t count, int nsq,
                  uint32_t* __restrict__ y, int* status) {
  namespace tc = pc2::tc;
  extern __shared__ __align__(1024) uint8_t smem[];
  const tc::Smem s = Core::smem_layout(smem);
  const uint32_t tmem = Core::setup(s, P.m);
  {
    tc::State st{0u, true};
    const size_t ntiles = (count + tc::kTileE - 1) / tc::kTileE;
    for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      size_t g = tile * tc::kTileE + threadIdx.x;
      const bool valid = g < count;
      if (!valid) g = count - 1;
      uint32_t a[kL];
#pragma unroll
      for (int j = 0; j < kL; ++j) a[j] = x[pc2::tiled_index(g, j, kL)];
      for (int it = 0; it < nsq; ++it) {
        Core::montsqr(a, s, tmem, P.m.n, st);
      }
      if (valid) {
#pragma unroll
        for (int j = 0; j < kL; ++j) y[pc2::tiled_index(g, j, kL)] = a[j];
      }
    }
    if (!st.ok && status) atomicOr(status, PC2_ST_TIMEOUT);
  }
  Core::teardown(tmem);
}

// ------------------------------------------------------------------ the integer-pipe kernel
// The same squarings with the library's CIOS product (one thread per
// element, the operand read from shared memory one word per row).
constexpr int kImadThreads = 128;
__global__ void __launch_bounds__(kImadThreads, 3)
    k_mont_sqr_imad(const __grid_constant__ SqrParams P, const uint32_t* __restrict__ x, size_t count, int nsq,
                    uint32_t* __restrict__ y) {
  extern __shared__ uint32_t bsh_all[];
  const pc2::Grp<1> g;
  const pc2::Col bsh{bsh_all + threadIdx.x, kImadThreads};
  for (size_t e0 = (size_t)blockIdx.x * kImadThreads; e0 < count; e0 += (size_t)gridDim.x * kImadThreads) {
    size_t e = e0 + threadIdx.x;
    const bool valid = e < count;
    if (!valid) e = count - 1;
    uint32_t a[kL];
#pragma unroll
    for (int j = 0; j < kL; ++j) a[j] = x[pc2::tiled_index(e, j, kL)];
    for (int it = 0; it < nsq; ++it) {
#pragma unroll
      for (int j = 0; j < kL; ++j) bsh[j] = a[j];
      pc2::mont_mul<kL, 1>(a, bsh.p, bsh.s, pc2::ParamN{P.m.n}, P.m.np0, g);
    }
    if (valid) {
#pragma unroll
      for (int j = 0; j < kL; ++j) y[pc2::tiled_index(e, j, kL)] = a[j];
    }
  }
}

}  // namespace

extern "C" int pc2_mont_sqr(pc2_ctx* ctx, const uint32_t* h_n, int limbs, const uint32_t* d_x, size_t count, int nsq,
                            int engine, uint32_t* d_y, pc2_stream_t stream) {
  if (!ctx || !h_n || (count && (!d_x || !d_y)) || nsq < 0) return PC2_EINVAL;
  if (limbs != kL) return PC2_EUNSUPPORTED;
  if (engine != PC2_ENGINE_IMAD && engine != PC2_ENGINE_TC) return PC2_EINVAL;
  if (!count) return PC2_OK;
  static thread_local SqrParams P;  // 17 KB: kept off the stack
  if (!pc2::tc::build_mod<kL>(h_n, P.m)) return PC2_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  if (engine == PC2_ENGINE_TC) {
    if (cudaFuncSetAttribute(k_mont_sqr_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, Core::kSmem) !=
        cudaSuccess)
      return PC2_ECUDA;
    const size_t tiles = (count + pc2::tc::kTileE - 1) / pc2::tc::kTileE;
    const size_t grid = tiles < (size_t)(2 * ctx->sms) ? tiles : (size_t)(2 * ctx->sms);
    k_mont_sqr_tc<<<(unsigned)grid, pc2::tc::kThreads, Core::kSmem, st>>>(P, d_x, count, nsq, d_y, ctx->status);
  } else {
    const size_t smem = (size_t)kL * kImadThreads * 4;
    if (cudaFuncSetAttribute(k_mont_sqr_imad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return PC2_ECUDA;
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mont_sqr_imad, kImadThreads, smem) != cudaSuccess ||
        per < 1)
      return PC2_ECUDA;
    const size_t blocks = (count + kImadThreads - 1) / kImadThreads;
    const size_t grid = blocks < (size_t)per * ctx->sms ? blocks : (size_t)per * ctx->sms;
    k_mont_sqr_imad<<<(unsigned)grid, kImadThreads, smem, st>>>(P, d_x, count, nsq, d_y);
  }
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}
