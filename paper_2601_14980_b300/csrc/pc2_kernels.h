// pc2_kernels.h -- internal launcher declarations (host side of the kernels).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/pc2.h"
#include "pc2_params.h"

namespace pc2 {

constexpr int kThreads = 128;  // threads per CTA of the modexp kernels

// Returns device scratch of at least `bytes` (owned by the context), or null.
typedef uint32_t* (*ScratchFn)(void* sctx, size_t bytes);

template <int Lh, int T>
int launch_enc_crt(const EncCrtParams<Lh>& P, const uint64_t* m64, const uint32_t* mwide, size_t count, uint32_t* out,
                   ScratchFn scratch_fn, void* sctx, int* status, int sms, cudaStream_t st, size_t base = 0);
template <int L2, int T>
int launch_enc_pub(const EncPubParams<L2>& P, const uint64_t* m64, const uint32_t* mwide, size_t count, uint32_t* out,
                   ScratchFn scratch_fn, void* sctx, int* status, int sms, cudaStream_t st);
template <int Lh, int T>
int launch_dec_crt(const DecParams<Lh>& P, const uint32_t* ct, size_t count, uint32_t* out, ScratchFn scratch_fn,
                   void* sctx, int sms, cudaStream_t st, size_t base = 0);
// The same operations with the two CRT halves of each element computed in
// parallel (T > 1): lower latency for batches that leave the GPU idle.
template <int Lh, int T>
int launch_enc_crt2(const EncCrtParams<Lh>& P, const uint64_t* m64, const uint32_t* mwide, size_t count, uint32_t* out,
                    ScratchFn scratch_fn, void* sctx, int* status, int sms, cudaStream_t st, size_t base = 0);
template <int Lh, int T>
int launch_dec_crt2(const DecParams<Lh>& P, const uint32_t* ct, size_t count, uint32_t* out, ScratchFn scratch_fn,
                    void* sctx, int sms, cudaStream_t st, size_t base = 0);
template <int Lh, int T>
int launch_dec_crt_fixed(const DecParams<Lh>& P, const uint32_t* ct, size_t count, uint32_t* out, uint32_t* scratch,
                         size_t scratch_words, int sms, cudaStream_t st);
template <int L2, int T>
int launch_hom_sum(const HomParams<L2>& P, size_t count, uint32_t* out, int sms, cudaStream_t st, size_t base = 0);
template <int L2, int T>
int launch_hom_scal(const HomParams<L2>& P, const uint32_t* ct, const uint64_t* k, size_t count, uint32_t* out,
                    ScratchFn scratch_fn, void* sctx, int sms, cudaStream_t st);
template <int L2, int T>
int launch_hom_scal_wide(const HomParams<L2>& P, const uint32_t* ct, const uint32_t* kw, size_t count, uint32_t* out,
                         ScratchFn scratch_fn, void* sctx, int sms, cudaStream_t st);
int launch_pack(const uint32_t* canon, size_t count, int Lc, uint32_t* tiled, int sms, cudaStream_t st);
int launch_unpack(const uint32_t* tiled, size_t count, int Lc, uint32_t* canon, int sms, cudaStream_t st);

// Resident CTAs per SM each kernel is compiled for: the register budget of
// 65536 / (128 * blocks) must hold two limb segments (three when the modulus
// segment lives in registers, T > 1) plus bookkeeping.  Measured on B300 with
// squaring loops: L=64, T=1 at 3 CTAs/SM (152 registers) reaches 18.0
// 32x32->64 products per clock per SM; L=96, T=2 at 2 CTAs 16.3; L=128, T=4 at
// 3 CTAs 17.0.  Keeping the budget
// tight stops the compiler from hoisting the modulus words (constant-bank
// operands) into registers.
constexpr int min_blocks(int L, int T) {
  const int S = L / T;
  const int regs = T == 1 ? 2 * S + 24 : 3 * S + 40;
  const int b = 65536 / (kThreads * regs);
  return b < 1 ? 1 : (b > 8 ? 8 : b);
}

// Lanes per element for each modulus width: the row core keeps a segment of
// the multiplicand and of the accumulator in registers (plus the modulus
// segment when T > 1); wider operands are split across lanes.
constexpr int lanes_for(int L) { return L <= 64 ? 1 : (L <= 96 ? 2 : 4); }

}  // namespace pc2
