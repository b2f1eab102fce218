// tc_mont.cu -- Montgomery squarings with the reduction on the tensor cores
// (pc2_mont_sqr, engine PC2_ENGINE_TC), beside the same squarings on the
// integer pipe (engine PC2_ENGINE_IMAD, the library's CIOS core).
//
// The paper multiplies big integers by transforms over small-base digit
// vectors and reduces by Barrett (Alg. 2, Eqs. (FFT)-(big_int_mul_2)).  The
// part of a modular product that is a dense contraction with an operand
// shared by all elements is the reduction: in separated operand scanning,
//   T = a b,  m = (T mod R) N' mod R,  U = (T + m N) / R   (N' = -N^-1 mod R),
// both m and m N multiply a per-element vector by the key's fixed N' or N.
// Written over 8-bit digits (x = sum_k x_k 256^k), the column sums
// C_j = sum_k x_k y_{j-k} are a product of an [elements x digits] matrix and
// a Toeplitz matrix of the fixed operand's digits.  Digits 0..255 are exact
// in bf16, and every column sum stays below 256 * 255^2 < 2^24, so the FP32
// accumulation of kind::f16 tcgen05.mma is exact.
//
// One CTA owns a tile of 128 elements (MMA M = 128, TMEM lane e = element e).
// Warps 0-3 hold one element per thread; warp 4 allocates TMEM and issues the
// MMAs.  Per squaring:
//   1. warps 0-3: T = a a by CIOS-style rows on the integer pipe (a in
//      registers, a's words read back from shared memory one per row); each
//      finished low word of T is written as four bf16 digits into the A tile.
//   2. warp 4: m-columns = A x Toeplitz(N') (columns 0..255) into TMEM.
//   3. warps 0-3: read the columns, propagate carries, write m's digits into
//      the A tile.
//   4. warp 4: Hi-columns 256..511 of m N (then, after they are read,
//      columns 240..255, which fix the carry out of the low half).
//   5. warps 0-3: U = T_hi + Hi + carry, then U - N if U >= N.
// The Toeplitz operand is the same for every K-slice of 16 digits once the
// slice's output columns are offset by 16 s, so each fixed operand is one
// small [rows x 16] matrix (8 KB for N', 8.5 KB for N) and slice s issues an
// MMA whose D starts 16 s columns further.  The A tile also stores each
// element's current value (word i in the first four bytes of the 8-byte slot
// its T word i overwrites after the row that reads it).
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "../../include/pc2.h"
#include "ctx.hpp"
#include "hostbn.hpp"
#include "mont.cuh"
#include "pc2_kernels.h"

namespace {

constexpr int kL = 64;               // limbs of the modulus (2048 bits)
constexpr int kD = 4 * kL;           // 8-bit digits per operand
constexpr int kTileE = 128;          // elements per tile (MMA M)
constexpr int kTcThreads = 160;      // warps 0-3 compute, warp 4 issues
constexpr int kB1Rows = 256;         // Toeplitz(N') rows: output columns 0..255 of a slice
constexpr int kB2Rows = 272;         // Toeplitz(N) rows: output columns 16 s .. 16 s + 271
constexpr int kSlab = kTileE * 16;   // bytes of one 8-digit K-block of the A tile
constexpr int kAbytes = (kD / 8) * kSlab;              // 64 KB
constexpr int kB1bytes = kB1Rows * 32;                 // 8 KB
constexpr int kB2bytes = kB2Rows * 32;                 // 8.5 KB
constexpr int kTcSmem = kAbytes + kB1bytes + kB2bytes + 64;
constexpr uint32_t kTmemCols = 256;
constexpr long kSpin = 1L << 20;     // bounded waits (a tile's MMAs take microseconds)

struct alignas(16) TcParams {
  uint32_t n[kL];                    // N
  uint16_t b1[kB1Rows * 16];         // Toeplitz(N') slice, bf16 bits, K-major no-swizzle layout
  uint16_t b2[kB2Rows * 16];         // Toeplitz(N) slice
  uint32_t np0;                      // -N^-1 mod 2^32 (IMAD engine)
};
static_assert(sizeof(TcParams) + 256 <= 32764, "parameter block too large");

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// Waits for phase `parity` of the barrier to complete; false after kSpin trips.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_addr(bar);
  for (long it = 0; it < kSpin; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// SMEM matrix descriptor, no swizzle, K-major: core matrices of 8 rows x 16 B,
// LBO = bytes between K-adjacent core matrices, SBO = bytes between 8-row groups.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: D f32, A and B bf16, both K-major, M = 128.
__host__ __device__ constexpr uint32_t idesc_bf16(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTileE >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void async_proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// Named barrier 1 between the compute warps (arrive) and the issuing warp (sync).
__device__ __forceinline__ void bar_arrive1() { asm volatile("bar.arrive 1, %0;" ::"n"(kTcThreads) : "memory"); }
__device__ __forceinline__ void bar_sync1() { asm volatile("bar.sync 1, %0;" ::"n"(kTcThreads) : "memory"); }

// 16 consecutive TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// An exact column sum (an integer below 2^24 held in f32) as an integer.
__device__ __forceinline__ uint64_t col(uint32_t bits) { return (uint64_t)__float2uint_rz(__uint_as_float(bits)); }

// The four digits of word w as bf16 (exact: 0..255), packed two per 32-bit word.
__device__ __forceinline__ uint2 word_digits(uint32_t w) {
  const uint32_t f0 = __float_as_uint(__uint2float_rn(w & 0xffu));
  const uint32_t f1 = __float_as_uint(__uint2float_rn((w >> 8) & 0xffu));
  const uint32_t f2 = __float_as_uint(__uint2float_rn((w >> 16) & 0xffu));
  const uint32_t f3 = __float_as_uint(__uint2float_rn(w >> 24));
  return make_uint2(__byte_perm(f0, f1, 0x7632), __byte_perm(f2, f3, 0x7632));
}

// Slot of word i of element e in the A tile (digits 4i..4i+3 of row e).
__device__ __forceinline__ uint32_t slot_off(int i, int e) { return (uint32_t)((i >> 1) * kSlab + e * 16 + (i & 1) * 8); }

// ------------------------------------------------------------------ the tensor-core kernel
__global__ void __launch_bounds__(kTcThreads, 2)
    k_mont_sqr_tc(const __grid_constant__ TcParams P, const uint32_t* __restrict__ x, size_t count, int nsq,
                  uint32_t* __restrict__ y, int* status) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* A = smem;
  uint8_t* B1 = smem + kAbytes;
  uint8_t* B2 = B1 + kB1bytes;
  uint64_t* bar = reinterpret_cast<uint64_t*>(B2 + kB2bytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // constants into shared memory (16-byte copies from the parameter block)
  {
    const uint4* s1 = reinterpret_cast<const uint4*>(P.b1);
    const uint4* s2 = reinterpret_cast<const uint4*>(P.b2);
    for (int i = threadIdx.x; i < kB1bytes / 16; i += kTcThreads) reinterpret_cast<uint4*>(B1)[i] = s1[i];
    for (int i = threadIdx.x; i < kB2bytes / 16; i += kTcThreads) reinterpret_cast<uint4*>(B2)[i] = s2[i];
  }
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  async_proxy_fence();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const size_t ntiles = (count + kTileE - 1) / kTileE;
  const uint32_t a_base = smem_addr(A), b1_base = smem_addr(B1), b2_base = smem_addr(B2);

  if (warp == 4) {
    // ---------------------------------------------------------------- issuer
    const bool leader = lane == 0;
    for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      for (int it = 0; it < nsq; ++it) {
        // (2) m-columns: slice s adds A[:, 16s..16s+15] x B1[0..255-16s] into columns 16s..255
        bar_sync1();
        tc_fence_after();
        if (leader) {
          for (int s = 0; s < kD / 16; ++s) {
            const int N = 256 - 16 * s;
            mma_bf16(tmem + 16 * s, sdesc(a_base + 2 * s * kSlab, kSlab, 128), sdesc(b1_base, kB1Rows * 16, 128),
                     idesc_bf16(N), s > 0);
          }
          mma_commit(bar);
        }
        __syncwarp();
        // (4a) columns 256..511 of m N into TMEM columns 0..255 (slice 15 first: it covers them all)
        bar_sync1();
        tc_fence_after();
        if (leader) {
          for (int s = kD / 16 - 1; s >= 0; --s) {
            const int N = 16 * s + 16, row0 = 256 - 16 * s;
            mma_bf16(tmem, sdesc(a_base + 2 * s * kSlab, kSlab, 128), sdesc(b2_base + row0 * 16, kB2Rows * 16, 128),
                     idesc_bf16(N), s != kD / 16 - 1);
          }
          mma_commit(bar);
        }
        __syncwarp();
        // (4b) columns 240..255 of m N into TMEM columns 0..15
        bar_sync1();
        tc_fence_after();
        if (leader) {
          for (int s = kD / 16 - 1; s >= 0; --s) {
            const int row0 = 240 - 16 * s;
            mma_bf16(tmem, sdesc(a_base + 2 * s * kSlab, kSlab, 128), sdesc(b2_base + row0 * 16, kB2Rows * 16, 128),
                     idesc_bf16(16), s != kD / 16 - 1);
          }
          mma_commit(bar);
        }
        __syncwarp();
      }
    }
  } else {
    // ---------------------------------------------------------------- compute warps
    const int e = threadIdx.x;                            // row of the tile = TMEM lane
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t phase = 0;
    bool ok = true;
    for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      size_t g = tile * kTileE + e;
      const bool valid = g < count;
      if (!valid) g = count - 1;
      uint32_t a[kL];
#pragma unroll
      for (int j = 0; j < kL; ++j) a[j] = x[pc2::tiled_index(g, j, kL)];
      for (int it = 0; it < nsq; ++it) {
        // the current value's words into their slots (read back one per row)
#pragma unroll
        for (int j = 0; j < kL; ++j) *reinterpret_cast<uint32_t*>(A + slot_off(j, e)) = a[j];
        // (1) T = a a: row i adds a * a_i; the finished low word becomes four digits
        uint32_t t[kL];
#pragma unroll
        for (int j = 0; j < kL; ++j) t[j] = 0u;
        uint32_t c0 = 0u, c1 = 0u, nz = 0u, top0 = 0u, top1 = 0u;
#pragma unroll 1
        for (int i = 0; i < kL; ++i) {
          const uint32_t bi = *reinterpret_cast<const uint32_t*>(A + slot_off(i, e));
          pc2::row_mac<kL>(t, c0, c1, pc2::RegA<kL>{a}, bi);
          const uint32_t w = t[0];
          nz |= w;
          top0 = i == kL - 2 ? w : top0;
          top1 = i == kL - 1 ? w : top1;
          *reinterpret_cast<uint2*>(A + slot_off(i, e)) = word_digits(w);
#pragma unroll
          for (int j = 0; j < kL - 1; ++j) t[j] = t[j + 1];
          t[kL - 1] = c0;
          c0 = c1;
          c1 = 0u;
        }
        // t = T_hi (T < N^2 < 2^4096, so nothing is left in c0)
        async_proxy_fence();
        tc_fence_before();
        bar_arrive1();
        ok = mbar_wait(bar, phase) && ok;
        phase ^= 1u;
        tc_fence_after();
        // (3) m = (sum_j C_j 256^j) mod R from columns 0..255
        {
          uint64_t carry = 0;
#pragma unroll 1
          for (int ch = 0; ch < 16; ++ch) {
            uint32_t r[16];
            tmem_ld16(lane_base + 16 * ch, r);
#pragma unroll
            for (int w = 0; w < 4; ++w) {
              const uint64_t v = carry + col(r[4 * w]) + (col(r[4 * w + 1]) << 8) + (col(r[4 * w + 2]) << 16) +
                                 (col(r[4 * w + 3]) << 24);
              carry = v >> 32;
              *reinterpret_cast<uint2*>(A + slot_off(4 * ch + w, e)) = word_digits((uint32_t)v);
            }
          }
        }
        async_proxy_fence();
        tc_fence_before();
        bar_arrive1();
        ok = mbar_wait(bar, phase) && ok;
        phase ^= 1u;
        tc_fence_after();
        // (5a) t += Hi = sum_j C_{256+j} 256^j
        uint32_t over = 0u;  // bit 2048 of the running sum
        {
          uint64_t carry = 0;
#pragma unroll
          for (int ch = 0; ch < 16; ++ch) {
            uint32_t r[16];
            tmem_ld16(lane_base + 16 * ch, r);
#pragma unroll
            for (int w = 0; w < 4; ++w) {
              const uint64_t v = carry + t[4 * ch + w] + col(r[4 * w]) + (col(r[4 * w + 1]) << 8) +
                                 (col(r[4 * w + 2]) << 16) + (col(r[4 * w + 3]) << 24);
              t[4 * ch + w] = (uint32_t)v;
              carry = v >> 32;
            }
          }
          over = (uint32_t)carry;
        }
        tc_fence_before();
        bar_arrive1();
        ok = mbar_wait(bar, phase) && ok;
        phase ^= 1u;
        tc_fence_after();
        // (5b) carry out of the low half: T_lo + Lo = c R with Lo = sum_{j<256} C_j 256^j.
        // Lo = F + c' R with F = (R - T_lo) mod R; c' = round((Lo - F) / R) from
        // columns 248..255 and the top 64 bits of F (error below 2^-39).
        {
          uint32_t r[16];
          tmem_ld16(lane_base, r);
          unsigned __int128 X = 0;
#pragma unroll
          for (int l = 15; l >= 8; --l) X = (X << 8) + (unsigned __int128)col(r[l]);
          const uint64_t ttop = ((uint64_t)top1 << 32) | top0;
          const unsigned __int128 Ftop = nz ? ((unsigned __int128)1 << 64) - ttop : 0;
          const __int128 d = (__int128)X - (__int128)Ftop + ((__int128)1 << 63);
          const uint64_t c = (uint64_t)(d >> 64) + (nz ? 1u : 0u);
          uint64_t v = (uint64_t)t[0] + (uint32_t)c;
          t[0] = (uint32_t)v;
          v = (v >> 32) + t[1] + (uint32_t)(c >> 32);
          t[1] = (uint32_t)v;
          v >>= 32;
#pragma unroll
          for (int j = 2; j < kL; ++j) {
            v += t[j];
            t[j] = (uint32_t)v;
            v >>= 32;
          }
          over += (uint32_t)v;
        }
        // U < 2N: subtract N when U >= N
        {
          uint32_t br;
          asm volatile("sub.cc.u32 %0, %1, %2;" : "=r"(a[0]) : "r"(t[0]), "r"(P.n[0]));
#pragma unroll
          for (int j = 1; j < kL; ++j) asm volatile("subc.cc.u32 %0, %1, %2;" : "=r"(a[j]) : "r"(t[j]), "r"(P.n[j]));
          asm volatile("subc.u32 %0, 0, 0;" : "=r"(br));
          const bool keep = over == 0u && br != 0u;
#pragma unroll
          for (int j = 0; j < kL; ++j) a[j] = keep ? t[j] : a[j];
        }
      }
      if (valid) {
#pragma unroll
        for (int j = 0; j < kL; ++j) y[pc2::tiled_index(g, j, kL)] = a[j];
      }
    }
    if (!ok && status) atomicOr(status, PC2_ST_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 4) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// ------------------------------------------------------------------ the integer-pipe kernel
// The same squarings with the library's CIOS product (one thread per
// element, the operand read from shared memory one word per row).
constexpr int kImadThreads = 128;
__global__ void __launch_bounds__(kImadThreads, 3)
    k_mont_sqr_imad(const __grid_constant__ TcParams P, const uint32_t* __restrict__ x, size_t count, int nsq,
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
      pc2::mont_mul<kL, 1>(a, bsh.p, bsh.s, pc2::ParamN{P.n}, P.np0, g);
    }
    if (valid) {
#pragma unroll
      for (int j = 0; j < kL; ++j) y[pc2::tiled_index(e, j, kL)] = a[j];
    }
  }
}

// ------------------------------------------------------------------ host set-up
uint16_t bf16_of_digit(uint32_t d) {
  float f = (float)d;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return (uint16_t)(u >> 16);  // exact: d < 256 needs 8 significant bits
}

// Toeplitz slice of a fixed operand's digits: row n, K column kk holds
// digit (n - kk) when 0 <= n - kk < 256, in the K-major no-swizzle layout
// (K-block kb of 8 columns is a [rows x 8] row-major slab).
void toeplitz_slice(const std::vector<uint32_t>& dig, int rows, uint16_t* out) {
  for (int n = 0; n < rows; ++n)
    for (int kk = 0; kk < 16; ++kk) {
      const int d = n - kk;
      const uint32_t v = (d >= 0 && d < kD) ? dig[d] : 0u;
      out[(kk / 8) * rows * 8 + n * 8 + (kk % 8)] = bf16_of_digit(v);
    }
}

std::vector<uint32_t> digits_of(const uint32_t* w) {
  std::vector<uint32_t> d(kD);
  for (int i = 0; i < kD; ++i) d[i] = (w[i / 4] >> (8 * (i % 4))) & 0xffu;
  return d;
}

int make_params(const uint32_t* h_n, TcParams& P) {
  if (!(h_n[0] & 1u)) return PC2_EINVAL;
  std::memcpy(P.n, h_n, sizeof(P.n));
  // N' = -N^-1 mod 2^2048 by Newton's iteration x <- x (2 - N x), doubling the correct bits
  std::vector<uint32_t> inv(kL, 0u), t(2 * kL), u(2 * kL);
  uint32_t x0 = 1u;
  for (int i = 0; i < 5; ++i) x0 *= 2u - h_n[0] * x0;  // mod 2^32
  inv[0] = x0;
  auto mullo = [&](const std::vector<uint32_t>& a, const uint32_t* b, std::vector<uint32_t>& r) {
    std::fill(r.begin(), r.end(), 0u);
    for (int i = 0; i < kL; ++i) {
      uint64_t c = 0;
      for (int j = 0; i + j < kL; ++j) {
        c += (uint64_t)a[i] * b[j] + r[i + j];
        r[i + j] = (uint32_t)c;
        c >>= 32;
      }
    }
  };
  for (int it = 0; it < 7; ++it) {  // 32 -> 4096 correct bits
    mullo(inv, h_n, t);             // t = N x
    // u = 2 - t mod R
    uint64_t br = 0;
    for (int j = 0; j < kL; ++j) {
      const uint64_t s = (j == 0 ? 2ull : 0ull), v = (uint64_t)t[j] + br;
      u[j] = (uint32_t)(s - v);
      br = s < v;
    }
    std::vector<uint32_t> un(u.begin(), u.begin() + kL);
    mullo(inv, un.data(), t);
    std::copy(t.begin(), t.begin() + kL, inv.begin());
  }
  // N' = R - inv
  std::vector<uint32_t> np(kL);
  uint64_t br = 0;
  for (int j = 0; j < kL; ++j) {
    const uint64_t v = (uint64_t)inv[j] + br;
    np[j] = (uint32_t)(0ull - v);
    br = v != 0;
  }
  P.np0 = np[0];
  toeplitz_slice(digits_of(np.data()), kB1Rows, P.b1);
  toeplitz_slice(digits_of(h_n), kB2Rows, P.b2);
  return PC2_OK;
}

}  // namespace

extern "C" int pc2_mont_sqr(pc2_ctx* ctx, const uint32_t* h_n, int limbs, const uint32_t* d_x, size_t count, int nsq,
                            int engine, uint32_t* d_y, pc2_stream_t stream) {
  if (!ctx || !h_n || (count && (!d_x || !d_y)) || nsq < 0) return PC2_EINVAL;
  if (limbs != kL) return PC2_EUNSUPPORTED;
  if (engine != PC2_ENGINE_IMAD && engine != PC2_ENGINE_TC) return PC2_EINVAL;
  if (!count) return PC2_OK;
  static thread_local TcParams P;  // 17 KB: kept off the stack
  int rc = make_params(h_n, P);
  if (rc != PC2_OK) return rc;
  const cudaStream_t st = (cudaStream_t)stream;
  if (engine == PC2_ENGINE_TC) {
    if (cudaFuncSetAttribute(k_mont_sqr_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem) != cudaSuccess)
      return PC2_ECUDA;
    const size_t tiles = (count + kTileE - 1) / kTileE;
    const size_t grid = tiles < (size_t)(2 * ctx->sms) ? tiles : (size_t)(2 * ctx->sms);
    k_mont_sqr_tc<<<(unsigned)grid, kTcThreads, kTcSmem, st>>>(P, d_x, count, nsq, d_y, ctx->status);
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
