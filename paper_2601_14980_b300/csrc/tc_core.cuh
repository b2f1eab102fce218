// tc_core.cuh -- Montgomery products of 2048-bit operands with the
// reduction on the tensor cores (tcgen05.mma, f16 digits, exact FP32
// column sums), for the modular exponentiations of libpc2.
//
// The part of a modular product that is a dense contraction with an operand
// shared by all elements is the reduction (the paper's Alg. 2 recasts
// big-integer products as low-bitwidth vector/matrix operations): in
// separated operand scanning,
//   T = a b,  m = (T mod R) N' mod R,  U = (T + m N) / R   (N' = -N^-1 mod R),
// and both m and m N multiply a per-element vector by the modulus' fixed N'
// or N.  Over 8-bit digits (x = sum_k x_k 256^k) the column sums
// C_j = sum_k x_k y_{j-k} are an [elements x digits] matrix times a
// Toeplitz matrix of the fixed operand's digits.  Digits 0..255 are exact in
// f16 and every column sum stays below 256 * 255^2 < 2^24, so the FP32
// accumulation of kind::f16 tcgen05.mma is exact.
//
// A CTA owns tiles of 128 elements (MMA M = 128, TMEM lane e = element e),
// one element per thread; warp 0 allocates 4L TMEM columns (L limbs, 4L
// digits) and thread 0 issues the MMAs.  No warp is set aside for the
// tensor cores: with four warps per CTA a thread may hold 255 registers at
// two CTAs per SM, enough for a 64-limb operand and its 128-word square.
// Below for L = 64.  One product a <- a b / R mod N:
//   1. T = a b by rows on the integer pipe (a in registers, b's word i read
//      from shared memory before row i); each finished low word of T is
//      written as four f16 digits into the A tile;
//   2. thread 0: m-columns = A x Toeplitz(N'), columns 0..255, into TMEM;
//   3. carries over the columns give m, whose digits go into the A tile;
//   4. thread 0: columns 256..511 of m N; after they are read, columns
//      240..255, which fix the carry out of the low half;
//   5. U = T_hi + Hi + carry, then U - N when U >= N.
// For every K-slice s of 16 digits the Toeplitz operand is the same
// [rows x 16] matrix once the slice's output columns start 16 s further, so
// a fixed operand costs one small slice (8 KB for N', 8.5 KB for N), and the
// A tile (64 KB) also holds each element's operand b: word i sits in the
// first four bytes of the 8-byte slot that T word i overwrites after row i.
// Shared memory per CTA: 81 KB at L = 64 (two CTAs per SM, 2 x 256 TMEM
// columns), 41 KB at L = 32 (four CTAs per SM, 4 x 128 columns).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "mont.cuh"
#include "pc2_tc.h"

namespace pc2 {
namespace tc {

constexpr int kTileE = 128;          // elements per tile (MMA M)
constexpr int kThreads = 128;        // one element per thread; thread 0 also issues the MMAs
constexpr int kSlab = kTileE * 16;   // bytes of one 8-digit K-block of the A tile
constexpr long kSpin = 1L << 20;     // bounded waits (a tile's MMAs take microseconds)

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// Waits for phase `parity` of the barrier; false after kSpin trips.
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
// SMEM matrix descriptor, no swizzle, K-major: LBO = bytes between K-adjacent
// 8x16-byte core matrices, SBO = bytes between 8-row groups.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: D f32, A and B f16 (format fields 0), both K-major, M = 128.
__host__ __device__ constexpr uint32_t idesc_f16(int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTileE >> 4) << 24);
}
__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void async_proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
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
// The four digits of word w as f16 (exact: 0..255), two per 32-bit word,
// without conversion instructions: byte b next to the exponent byte 0x64
// is the f16 number 1024 + b, and one packed subtraction leaves b.
__device__ __forceinline__ uint2 word_digits(uint32_t w) {
  const uint32_t x0 = __byte_perm(w, 0x64646464u, 0x4140), x1 = __byte_perm(w, 0x64646464u, 0x4342);
  uint32_t d0, d1;
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(d0) : "r"(x0), "r"(0x64006400u));
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(d1) : "r"(x1), "r"(0x64006400u));
  return make_uint2(d0, d1);
}
// Byte offset of word i of element e in the A tile (digits 4i..4i+3 of row e).
__device__ __forceinline__ uint32_t slot_off(int i, int e) { return (uint32_t)((i >> 1) * kSlab + e * 16 + (i & 1) * 8); }

// Shared-memory layout and TMEM of one CTA.
struct Smem {
  uint8_t* A;
  uint8_t* B1;
  uint8_t* B2;
  uint64_t* bar;
  uint32_t* tmem_slot;
};
// Per-thread state of the compute side.
struct State {
  uint32_t phase;
  bool ok;
};

// Result of the product phase: t = T_hi (words 64..127 of T), the low words
// already in the A tile as digits; nz = (T_lo != 0); top = words 62, 63 of T.
struct Prod {
  uint32_t nz, top0, top1;
};

// The L-limb product (L = 32 or 64): digits, tile and TMEM sizes, and every
// step that depends on them.
template <int L>
struct Core {
  static constexpr int kL = L;
  static constexpr int kD = 4 * L;              // 8-bit digits per operand
  static constexpr int kB1Rows = kD;            // Toeplitz(N') slice rows: output columns 0 .. kD-1
  static constexpr int kB2Rows = kD + 16;       // Toeplitz(N) slice rows: output columns 16 s .. 16 s + kD + 15
  static constexpr int kAbytes = (kD / 8) * kSlab;
  static constexpr int kB1bytes = kB1Rows * 32;
  static constexpr int kB2bytes = kB2Rows * 32;
  static constexpr int kSmem = kAbytes + kB1bytes + kB2bytes + 64;
  static constexpr uint32_t kTmemCols = kD;     // a power of two for L = 32, 64

static __device__ __forceinline__ Smem smem_layout(uint8_t* base) {
  Smem s;
  s.A = base;
  s.B1 = base + kAbytes;
  s.B2 = s.B1 + kB1bytes;
  s.bar = reinterpret_cast<uint64_t*>(s.B2 + kB2bytes);
  s.tmem_slot = reinterpret_cast<uint32_t*>(s.bar + 1);
  return s;
}

// Start of the kernel (all threads): the Toeplitz slices into shared memory,
// the barrier, kD TMEM columns.  Returns the TMEM base address.
static __device__ __forceinline__ uint32_t setup(const Smem& s, const Mod<L>& M) {
  const uint4* s1 = reinterpret_cast<const uint4*>(M.b1);
  const uint4* s2 = reinterpret_cast<const uint4*>(M.b2);
  for (int i = threadIdx.x; i < kB1bytes / 16; i += kThreads) reinterpret_cast<uint4*>(s.B1)[i] = s1[i];
  for (int i = threadIdx.x; i < kB2bytes / 16; i += kThreads) reinterpret_cast<uint4*>(s.B2)[i] = s2[i];
  if (threadIdx.x == 0) {
    mbar_init(s.bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s.tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  async_proxy_fence();
  fence_before();
  __syncthreads();
  fence_after();
  return *s.tmem_slot;
}

// End of the kernel (all threads): release the TMEM columns.
static __device__ __forceinline__ void teardown(uint32_t tmem) {
  fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// The three MMA groups of a product (thread 0).
// m-columns: slice k adds A[:, 16k..16k+15] x B1[0..kD-1-16k] into columns 16k..kD-1.
static __device__ __forceinline__ void issue_m(const Smem& s, uint32_t tmem) {
  const uint32_t a_base = smem_addr(s.A), b1_base = smem_addr(s.B1);
  for (int k = 0; k < kD / 16; ++k)
    mma_f16(tmem + 16 * k, sdesc(a_base + 2 * k * kSlab, kSlab, 128), sdesc(b1_base, kB1Rows * 16, 128),
             idesc_f16(kD - 16 * k), k > 0);
}
// Columns kD..2kD-1 of m N into TMEM columns 0..kD-1 (the last slice first: it covers them all).
static __device__ __forceinline__ void issue_hi(const Smem& s, uint32_t tmem) {
  const uint32_t a_base = smem_addr(s.A), b2_base = smem_addr(s.B2);
  for (int k = kD / 16 - 1; k >= 0; --k)
    mma_f16(tmem, sdesc(a_base + 2 * k * kSlab, kSlab, 128), sdesc(b2_base + (kD - 16 * k) * 16, kB2Rows * 16, 128),
             idesc_f16(16 * k + 16), k != kD / 16 - 1);
}
// Columns kD-16..kD-1 of m N into TMEM columns 0..15.
static __device__ __forceinline__ void issue_carry(const Smem& s, uint32_t tmem) {
  const uint32_t a_base = smem_addr(s.A), b2_base = smem_addr(s.B2);
  for (int k = kD / 16 - 1; k >= 0; --k)
    mma_f16(tmem, sdesc(a_base + 2 * k * kSlab, kSlab, 128),
             sdesc(b2_base + (kD - 16 - 16 * k) * 16, kB2Rows * 16, 128), idesc_f16(16), k != kD / 16 - 1);
}
// Hands the A tile and TMEM to the tensor cores for one group: every
// thread's shared-memory writes and TMEM reads are ordered before the
// barrier, thread 0 issues the group and commits it, and every thread
// waits (bounded) for its completion.
template <class Issue>
static __device__ __forceinline__ void mma_step(const Smem& s, uint32_t tmem, State& st, Issue issue) {
  async_proxy_fence();
  fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    fence_after();
    issue(s, tmem);
    mma_commit(s.bar);
  }
  st.ok = mbar_wait(s.bar, st.phase) && st.ok;
  st.phase ^= 1u;
  __syncwarp();
  fence_after();
}

// Product phase of a general product, element e = threadIdx.x: T = a b with
// b's words in their slots of the A tile (write_b_*), by rows on the integer
// pipe; each finished low word of T becomes four digits in its slot.
static __device__ __forceinline__ Prod product_rows(const uint32_t (&a)[kL], uint32_t (&t)[kL], const Smem& s) {
  const int e = threadIdx.x;
  uint8_t* A = s.A;
#pragma unroll
  for (int j = 0; j < kL; ++j) t[j] = 0u;
  Prod pr{0u, 0u, 0u};
#pragma unroll 4
  for (int i = 0; i < kL; ++i) {
    const uint32_t bi = *reinterpret_cast<const uint32_t*>(A + slot_off(i, e));
    // t += a bi: each step a bi_j + t_j + c < 2^64, one wide product and a
    // 64-bit add, the carry in a register (no carry-flag chain)
    uint32_t c = 0u;
#pragma unroll
    for (int j = 0; j < kL; ++j) {
      const uint64_t p = (uint64_t)a[j] * bi + t[j] + c;
      t[j] = (uint32_t)p;
      c = (uint32_t)(p >> 32);
    }
    const uint32_t w = t[0];
    pr.nz |= w;
    pr.top0 = i == kL - 2 ? w : pr.top0;
    pr.top1 = i == kL - 1 ? w : pr.top1;
    *reinterpret_cast<uint2*>(A + slot_off(i, e)) = word_digits(w);
#pragma unroll
    for (int j = 0; j < kL - 1; ++j) t[j] = t[j + 1];
    t[kL - 1] = c;
  }
  return pr;  // T < N^2 < 2^4096: nothing is left above t
}

// Row i of the squaring's cross products: C += a_i (a_{i+1} .. a_63) at
// positions 2i+1 .. i+63 and the row's carry word at i+64 (no earlier row
// reaches it), one wide product and a 64-bit add per step; positions up to
// 2i+2 are then final, and those below 64 are parked in their slots of the
// A tile.
template <int I>
static __device__ __forceinline__ void sqr_row(uint32_t (&C)[2 * kL], const uint32_t (&a)[kL], uint8_t* A, int e) {
  uint32_t c = 0u;
#pragma unroll
  for (int j = I + 1; j < kL; ++j) {
    const uint64_t p = (uint64_t)a[I] * a[j] + C[I + j] + c;
    C[I + j] = (uint32_t)p;
    c = (uint32_t)(p >> 32);
  }
  C[I + kL] = c;
  if constexpr (2 * I + 1 < kL) *reinterpret_cast<uint32_t*>(A + slot_off(2 * I + 1, e)) = C[2 * I + 1];
  if constexpr (2 * I + 2 < kL) *reinterpret_cast<uint32_t*>(A + slot_off(2 * I + 2, e)) = C[2 * I + 2];
}
template <int I, int END>
static __device__ __forceinline__ void sqr_rows(uint32_t (&C)[2 * kL], const uint32_t (&a)[kL], uint8_t* A, int e) {
  if constexpr (I < END) {
    sqr_row<I>(C, a, A, e);
    sqr_rows<I + 1, END>(C, a, A, e);
  }
}
// Product phase of a squaring, element e = threadIdx.x: T = a^2 = 2 C + D
// with C = sum_{i<j} a_i a_j 2^(32(i+j)) (rows of shrinking length, fully
// unrolled, a in registers) and D = sum_i a_i^2 2^(64 i): 2080 word products
// instead of 4096.  Finished words of C below 64 wait in their slots of the
// A tile; one pass then doubles C, adds D and writes the low words' digits.
static __device__ __forceinline__ Prod product_sqr(const uint32_t (&a)[kL], uint32_t (&t)[kL], const Smem& s) {
  const int e = threadIdx.x;
  uint8_t* A = s.A;
  uint32_t C[2 * kL];
#pragma unroll
  for (int k = 0; k < kL + 2; ++k) C[k] = 0u;
  C[2 * kL - 1] = 0u;
  Prod pr{0u, 0u, 0u};
  uint32_t prev = 0u;
  uint64_t carry = 0;
  // T_k = 2 C_k + D_k + carry, for k in [K0, K1)
  auto pass = [&](auto k0, auto k1) {
#pragma unroll
    for (int k = decltype(k0)::value; k < decltype(k1)::value; ++k) {
      const uint32_t ck = k == 0 ? 0u : (k < kL ? *reinterpret_cast<const uint32_t*>(A + slot_off(k, e)) : C[k]);
      const uint32_t dbl = (ck << 1) | (prev >> 31);
      prev = ck;
      const uint32_t ai = a[k >> 1];
      const uint32_t dk = (k & 1) ? __umulhi(ai, ai) : ai * ai;
      const uint64_t v = carry + dbl + dk;
      const uint32_t w = (uint32_t)v;
      carry = v >> 32;
      if (k < kL) {
        pr.nz |= w;
        if (k == kL - 2) pr.top0 = w;
        if (k == kL - 1) pr.top1 = w;
        *reinterpret_cast<uint2*>(A + slot_off(k, e)) = word_digits(w);
      } else {
        t[k - kL] = w;
      }
    }
  };
  // rows 0..31 finish every position below 65; the low half's pass then
  // frees a_0 .. a_31 before the remaining rows
  sqr_rows<0, kL / 2>(C, a, A, e);
  pass(std::integral_constant<int, 0>(), std::integral_constant<int, kL>());
  sqr_rows<kL / 2, kL - 1>(C, a, A, e);
  pass(std::integral_constant<int, kL>(), std::integral_constant<int, 2 * kL>());
  return pr;
}

// Reduction phase, element e = threadIdx.x: from T (t = T_hi, the low words'
// digits in the A tile) to a = T / R mod N with the tensor cores.
static __device__ __forceinline__ void reduce(uint32_t (&a)[kL], uint32_t (&t)[kL], const Prod& pr, const Smem& s,
                                       uint32_t tmem, const uint32_t* n, State& st) {
  const int e = threadIdx.x;
  const int warp = e >> 5;
  const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
  uint8_t* A = s.A;
  mma_step(s, tmem, st, [](const Smem& s_, uint32_t t_) { issue_m(s_, t_); });
  // 3. m = (sum_j C_j 256^j) mod R from columns 0..kD-1; its digits into the A tile
  {
    uint64_t carry = 0;
#pragma unroll 1
    for (int ch = 0; ch < kD / 16; ++ch) {
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
  mma_step(s, tmem, st, [](const Smem& s_, uint32_t t_) { issue_hi(s_, t_); });
  // 5a. t += Hi = sum_j C_{kD+j} 256^j
  uint32_t over = 0u;  // bit 32 L of the running sum
  {
    uint64_t carry = 0;
#pragma unroll
    for (int ch = 0; ch < kD / 16; ++ch) {
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
  mma_step(s, tmem, st, [](const Smem& s_, uint32_t t_) { issue_carry(s_, t_); });
  // 5b. carry out of the low half: T_lo + Lo = c R, Lo = sum_{j<kD} C_j 256^j.
  // Lo = F + c' R with F = (R - T_lo) mod R; c' = round((Lo - F) / R) from
  // the top 8 columns and the top 64 bits of F (error below 2^-39).
  {
    uint32_t r[16];
    tmem_ld16(lane_base, r);
    unsigned __int128 X = 0;
#pragma unroll
    for (int l = 15; l >= 8; --l) X = (X << 8) + (unsigned __int128)col(r[l]);
    const uint64_t ttop = ((uint64_t)pr.top1 << 32) | pr.top0;
    const unsigned __int128 Ftop = pr.nz ? ((unsigned __int128)1 << 64) - ttop : 0;
    const __int128 d = (__int128)X - (__int128)Ftop + ((__int128)1 << 63);
    const uint64_t c = (uint64_t)(d >> 64) + (pr.nz ? 1u : 0u);
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
  uint32_t br;
  asm volatile("sub.cc.u32 %0, %1, %2;" : "=r"(a[0]) : "r"(t[0]), "r"(n[0]));
#pragma unroll
  for (int j = 1; j < kL; ++j) asm volatile("subc.cc.u32 %0, %1, %2;" : "=r"(a[j]) : "r"(t[j]), "r"(n[j]));
  asm volatile("subc.u32 %0, 0, 0;" : "=r"(br));
  const bool keep = over == 0u && br != 0u;
#pragma unroll
  for (int j = 0; j < kL; ++j) a[j] = keep ? t[j] : a[j];
}


// a <- a b / R mod N, b's words already in their slots (write_b_*).
static __device__ __forceinline__ void montmul(uint32_t (&a)[kL], const Smem& s, uint32_t tmem, const uint32_t* n,
                                        State& st) {
  uint32_t t[kL];
  const Prod pr = product_rows(a, t, s);
  reduce(a, t, pr, s, tmem, n, st);
}
// a <- a^2 / R mod N (no operand slots needed).
static __device__ __forceinline__ void montsqr(uint32_t (&a)[kL], const Smem& s, uint32_t tmem, const uint32_t* n,
                                        State& st) {
  uint32_t t[kL];
  const Prod pr = product_sqr(a, t, s);
  reduce(a, t, pr, s, tmem, n, st);
}

// b = the thread's own a (a squaring).
static __device__ __forceinline__ void write_b_self(const Smem& s, const uint32_t (&a)[kL]) {
#pragma unroll
  for (int j = 0; j < kL; ++j) *reinterpret_cast<uint32_t*>(s.A + slot_off(j, threadIdx.x)) = a[j];
}
// b = word j at src[j * stride] (a table entry in global memory).
static __device__ __forceinline__ void write_b_global(const Smem& s, const uint32_t* src, size_t stride) {
#pragma unroll 8
  for (int j = 0; j < kL; ++j)
    *reinterpret_cast<uint32_t*>(s.A + slot_off(j, threadIdx.x)) = src[(size_t)j * stride];
}

};

}  // namespace tc
}  // namespace pc2
