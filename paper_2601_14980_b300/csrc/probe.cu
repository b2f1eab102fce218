// probe.cu -- throughput probe of the integer multiplier (pc2_probe_mul).
//
// The modular exponentiations are bound by the 32-bit multiply pipe, so
// their roofline needs its measured rate on this GPU, not a nominal unit
// count.  Each kernel below keeps several independent accumulators per
// thread (enough instruction-level parallelism that latency is hidden at
// full occupancy) and counts the operations it issues:
//   LO    mad.lo.u32            low half of a 32x32 product, plus an add
//   HI    mad.hi.u32            high half
//   WIDE  mad.wide.u32          a whole 32x32->64 product plus a 64-bit add
//   LOHI  mad.lo + mad.hi       a 32x32->64 product from two halves
// Each step feeds the accumulator back into the multiplier, so no product
// is loop-invariant (the assembler would otherwise hoist it).
//   DADD  add.rn.f64 (the FP64 pipe the z/v update of the ADMM uses)
//   ROW   the carry-chained row of a 64-limb Montgomery product
//         (mad.lo.cc / madc.lo.cc, then mad.hi.cc / madc.hi.cc); one product
//         per limb and row.
//   ROWW  the same rows in the wide form of the library's products (both
//         engines): t_j + a_j b + c as one 32x32->64 product and a 64-bit
//         add, the carry in a register.
// Cycles come from clock64 around the loop (max over CTAs), time from CUDA
// events around the launch.
#include <cuda_runtime.h>

#include "../../include/pc2.h"
#include "mont.cuh"

namespace {

// t[0..63], (c0, c1) += a * b with carry-flag chains: the low halves of the
// 32x32 products (mad.lo.cc / madc.lo.cc), then the high halves.
__device__ __forceinline__ void cc_row(uint32_t (&t)[64], uint32_t& c0, uint32_t& c1, const uint32_t (&a)[64],
                                       uint32_t b) {
  pc2::mad_lo_cc(t[0], a[0], b);
#pragma unroll
  for (int j = 1; j < 64; ++j) pc2::madc_lo_cc(t[j], a[j], b);
  pc2::addc_cc_z(c0);
  pc2::addc_z(c1);
  pc2::mad_hi_cc(t[1], a[0], b);
#pragma unroll
  for (int j = 1; j < 63; ++j) pc2::madc_hi_cc(t[j + 1], a[j], b);
  pc2::madc_hi_cc(c0, a[63], b);
  pc2::addc_z(c1);
}

constexpr int kProbeThreads = 128;
constexpr int kIlp = 8;

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads, KIND == PC2_PROBE_ROW || KIND == PC2_PROBE_ROWW ? 3 : 8) k_probe(uint32_t seed, int iters, uint32_t* sink,
                                                         long long* cycles) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t b = seed * 2654435761u + tid;
  long long t0 = 0;
  uint32_t fold = 0;
  if constexpr (KIND == PC2_PROBE_ROW) {
    uint32_t a[64], t[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) {
      a[j] = b ^ (j * 0x9e3779b9u);
      t[j] = j;
    }
    uint32_t c0 = 0, c1 = 0;
    __syncthreads();
    t0 = clock64();
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll 1
      for (int r = 0; r < 64; ++r) {
        cc_row(t, c0, c1, a, b + r);
      }
    }
#pragma unroll
    for (int j = 0; j < 64; ++j) fold ^= t[j];
    fold ^= c0 ^ c1;
  } else if constexpr (KIND == PC2_PROBE_ROWW) {
    uint32_t a[64], t[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) {
      a[j] = b ^ (j * 0x9e3779b9u);
      t[j] = j;
    }
    uint32_t top = 0;
    __syncthreads();
    t0 = clock64();
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll 1
      for (int r = 0; r < 64; ++r) {
        const uint32_t br = b + r;
        uint32_t c = 0u;
#pragma unroll
        for (int j = 0; j < 64; ++j) {
          const uint64_t p = (uint64_t)a[j] * br + t[j] + c;
          t[j] = (uint32_t)p;
          c = (uint32_t)(p >> 32);
        }
        top ^= c;
      }
    }
#pragma unroll
    for (int j = 0; j < 64; ++j) fold ^= t[j];
    fold ^= top;
  } else if constexpr (KIND == PC2_PROBE_DADD) {
    // x <- x + y in IEEE double (the z/v update's arithmetic); y changes the
    // low bits so nothing is constant
    double x[kIlp];
#pragma unroll
    for (int k = 0; k < kIlp; ++k) x[k] = (double)(b + k);
    const double y = 1.0 + (double)(b & 7u) * 0x1p-40;
    __syncthreads();
    t0 = clock64();
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < 16; ++u) {
#pragma unroll
        for (int k = 0; k < kIlp; ++k) asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(x[k]) : "d"(y));
      }
    }
#pragma unroll
    for (int k = 0; k < kIlp; ++k) fold ^= (uint32_t)__double2loint(x[k]);
  } else if constexpr (KIND == PC2_PROBE_WIDE) {
    // x <- lo(x) * b + x: the multiplier input changes every step
    uint64_t x[kIlp];
#pragma unroll
    for (int k = 0; k < kIlp; ++k) x[k] = b + k;
    __syncthreads();
    t0 = clock64();
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < 16; ++u) {
#pragma unroll
        for (int k = 0; k < kIlp; ++k)
          asm volatile("{\n .reg .b32 lo, hi;\n mov.b64 {lo, hi}, %0;\n mad.wide.u32 %0, lo, %1, %0;\n}\n"
                       : "+l"(x[k])
                       : "r"(b));
      }
    }
#pragma unroll
    for (int k = 0; k < kIlp; ++k) fold ^= (uint32_t)x[k] ^ (uint32_t)(x[k] >> 32);
  } else {
    // LO: x <- lo(x b) + c; HI: y <- hi(y b) + c; LOHI: both halves of x b
    uint32_t x[kIlp], y[kIlp];
#pragma unroll
    for (int k = 0; k < kIlp; ++k) {
      x[k] = b + k;
      y[k] = b ^ k;
    }
    const uint32_t c = b | 1u;
    __syncthreads();
    t0 = clock64();
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < 16; ++u) {
#pragma unroll
        for (int k = 0; k < kIlp; ++k) {
          if constexpr (KIND == PC2_PROBE_LO)
            asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[k]) : "r"(b), "r"(c));
          if constexpr (KIND == PC2_PROBE_HI)
            asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(y[k]) : "r"(b), "r"(c));
          if constexpr (KIND == PC2_PROBE_LOHI)
            asm volatile("{\n .reg .b32 l;\n mad.lo.u32 l, %0, %2, %1;\n mad.hi.u32 %1, %0, %2, %1;\n mov.b32 %0, l;\n}\n"
                         : "+r"(x[k]), "+r"(y[k])
                         : "r"(b));
        }
      }
    }
#pragma unroll
    for (int k = 0; k < kIlp; ++k) fold ^= x[k] ^ y[k];
  }
  const long long t1 = clock64();
  __syncthreads();
  if (fold == 0x12345678u) sink[tid] = fold;  // keeps the work observable
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

template <int KIND>
double ops_per_thread(int iters) {
  if constexpr (KIND == PC2_PROBE_ROW || KIND == PC2_PROBE_ROWW) return (double)iters * 64.0 * 64.0;
  else return (double)iters * 16.0 * kIlp;
}

template <int KIND>
int run(int sms, int blocks_per_sm, int iters, cudaStream_t st, double* ops, double* ms, double* cycles) {
  auto kern = k_probe<KIND>;
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kProbeThreads, 0) != cudaSuccess) return PC2_ECUDA;
  if (blocks_per_sm < 1 || blocks_per_sm > per) return PC2_EINVAL;  // every CTA must be resident
  const int grid = blocks_per_sm * sms;
  uint32_t* sink = nullptr;
  long long* cyc = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = PC2_OK;
  if (cudaMalloc(&sink, (size_t)grid * kProbeThreads * 4) != cudaSuccess ||
      cudaMalloc(&cyc, (size_t)grid * sizeof(long long)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    rc = PC2_ENOMEM;
  } else {
    cudaEventRecord(e0, st);
    kern<<<grid, kProbeThreads, 0, st>>>(0x5eedu, iters, sink, cyc);
    cudaEventRecord(e1, st);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      rc = PC2_ECUDA;
    } else {
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      long long* h = new long long[grid];
      if (cudaMemcpy(h, cyc, (size_t)grid * sizeof(long long), cudaMemcpyDeviceToHost) != cudaSuccess) rc = PC2_ECUDA;
      long long mx = 0;
      for (int i = 0; i < grid; ++i) mx = h[i] > mx ? h[i] : mx;
      delete[] h;
      *ops = ops_per_thread<KIND>(iters) * (double)grid * kProbeThreads;
      *ms = t;
      *cycles = (double)mx;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (cyc) cudaFree(cyc);
  return rc;
}

}  // namespace

extern "C" int pc2_probe_mul(int device, int kind, int blocks_per_sm, int iters, pc2_stream_t stream, double* ops,
                             double* ms, double* cycles, int* sms_out) {
  if (!ops || !ms || !cycles || iters < 1) return PC2_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return PC2_ECUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return PC2_ECUDA;
  if (sms_out) *sms_out = sms;
  const cudaStream_t st = (cudaStream_t)stream;
  switch (kind) {
    case PC2_PROBE_LO: return run<PC2_PROBE_LO>(sms, blocks_per_sm, iters, st, ops, ms, cycles);
    case PC2_PROBE_HI: return run<PC2_PROBE_HI>(sms, blocks_per_sm, iters, st, ops, ms, cycles);
    case PC2_PROBE_WIDE: return run<PC2_PROBE_WIDE>(sms, blocks_per_sm, iters, st, ops, ms, cycles);
    case PC2_PROBE_LOHI: return run<PC2_PROBE_LOHI>(sms, blocks_per_sm, iters, st, ops, ms, cycles);
    case PC2_PROBE_ROW: return run<PC2_PROBE_ROW>(sms, blocks_per_sm, iters, st, ops, ms, cycles);
    case PC2_PROBE_DADD: return run<PC2_PROBE_DADD>(sms, blocks_per_sm, iters, st, ops, ms, cycles);
    case PC2_PROBE_ROWW: return run<PC2_PROBE_ROWW>(sms, blocks_per_sm, iters, st, ops, ms, cycles);
    default: return PC2_EINVAL;
  }
}
