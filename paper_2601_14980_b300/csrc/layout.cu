#include <cuda_runtime.h>
#include "mont.cuh"
#include "pc2_kernels.h"

namespace pc2 {

// ------------------------------------------------------------------ layout conversion
__global__ void k_pack(const uint32_t* __restrict__ canon, size_t count, int Lc, uint32_t* __restrict__ tiled) {
  const size_t total = count * (size_t)Lc;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t e = i / (size_t)Lc;
    const int j = (int)(i % (size_t)Lc);
    tiled[tiled_index(e, j, Lc)] = canon[i];
  }
}
__global__ void k_unpack(const uint32_t* __restrict__ tiled, size_t count, int Lc, uint32_t* __restrict__ canon) {
  const size_t total = count * (size_t)Lc;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t e = i / (size_t)Lc;
    const int j = (int)(i % (size_t)Lc);
    canon[i] = tiled[tiled_index(e, j, Lc)];
  }
}


int launch_pack(const uint32_t* canon, size_t count, int Lc, uint32_t* tiled, int sms, cudaStream_t st) {
  k_pack<<<sms * 8, 256, 0, st>>>(canon, count, Lc, tiled);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}
int launch_unpack(const uint32_t* tiled, size_t count, int Lc, uint32_t* canon, int sms, cudaStream_t st) {
  k_unpack<<<sms * 8, 256, 0, st>>>(tiled, count, Lc, canon);
  return cudaGetLastError() == cudaSuccess ? PC2_OK : PC2_ECUDA;
}

}  // namespace pc2
