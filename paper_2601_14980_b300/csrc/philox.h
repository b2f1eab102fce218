// philox.h -- Philox4x32-10 counter-based generator (Salmon, Moraes, Dror,
// Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11), host and
// device.  Used for the encryption randomness r of Eq. (itq1) and for the
// deterministic key generator.
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define PC2_HD __host__ __device__ __forceinline__
#else
#define PC2_HD inline
#endif

namespace pc2 {

struct U4 { uint32_t x, y, z, w; };

PC2_HD uint32_t philox_mulhi(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

// Ten rounds; the key is bumped by the Weyl constants before rounds 2..10.
PC2_HD U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t h0 = philox_mulhi(0xD2511F53u, c.x), l0 = 0xD2511F53u * c.x;
    const uint32_t h1 = philox_mulhi(0xCD9E8D57u, c.z), l1 = 0xCD9E8D57u * c.z;
    c = U4{h1 ^ c.y ^ k0, l1, h0 ^ c.w ^ k1, l0};
  }
  return c;
}

// Block j of the draw for element e: counter (j, e_lo, e_hi, stream), key (seed_lo, seed_hi).
PC2_HD U4 r_block(uint64_t seed, uint32_t stream, uint64_t e, uint32_t j) {
  return philox4x32_10(U4{j, (uint32_t)e, (uint32_t)(e >> 32), stream}, (uint32_t)seed, (uint32_t)(seed >> 32));
}

}  // namespace pc2
