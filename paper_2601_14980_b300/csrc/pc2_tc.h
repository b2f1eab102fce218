// pc2_tc.h -- host-side declarations of the tensor-core Montgomery path
// (tc_core.cuh, tc_paillier.cu): the per-modulus constant block and the
// launchers of encryption and decryption at 2048-bit n.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "pc2_kernels.h"
#include "pc2_params.h"

namespace pc2 {
namespace tc {

// A modulus N of L words (L = 32 or 64) with its two Toeplitz slices (f16
// bits, K-major, no swizzle: K-block kb of 8 columns is a [rows x 8]
// row-major slab).
template <int L>
struct alignas(16) Mod {
  uint32_t n[L];
  uint16_t b1[4 * L * 16];        // digits of N' = -N^-1 mod 2^(32 L); rows 0 .. 4L-1
  uint16_t b2[(4 * L + 16) * 16];  // digits of N; rows 0 .. 4L+15
  uint32_t np0;                   // -N^-1 mod 2^32
  uint32_t pad_[3];
};

// Builds the block of an odd N (host).  False for an even N.
template <int L>
bool build_mod(const uint32_t* n, Mod<L>& M);

}  // namespace tc

// The blocks of p^2 and q^2 (64 words) and of p and q (32 words) of a
// 2048-bit key.
struct TcKeyMods {
  tc::Mod<64> p2, q2;
  tc::Mod<32> p, q;
};

// Key-owner encryption / CRT decryption at 2048-bit n with the full-width
// powers on the tensor cores; same arguments and results as launch_enc_crt /
// launch_dec_crt.
// ev (optional): five events recorded on `st` around the four launches
// (before set-up, after set-up, after each power, after the finish).
int launch_enc_crt_tc(const EncCrtParams<64>& P, const TcKeyMods& K, const uint64_t* m64, const uint32_t* mwide,
                      size_t count, uint32_t* out, ScratchFn scratch_fn, void* sctx, int* status, int sms,
                      cudaStream_t st, size_t base, cudaEvent_t* ev);
int launch_dec_crt_tc(const DecParams<64>& P, const TcKeyMods& K, const uint32_t* ct, size_t count, uint32_t* out,
                      ScratchFn scratch_fn, void* sctx, int* status, int sms, cudaStream_t st, size_t base,
                      cudaEvent_t* ev);

}  // namespace pc2
