// ctx.hpp -- the library context (internal layout) and internal helpers
// shared by the C-ABI translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>

#include "../../include/pc2.h"

struct pc2_ctx {
  int device = 0;
  int sms = 0;
  uint32_t* scratch = nullptr;
  size_t scratch_bytes = 0;
  int* status = nullptr;  // device word of PC2_ST_* bits
  int window = 0;         // 0 = automatic
  int lanes = 0;          // 0 = automatic (tuned table, else fill heuristic)
  // autotuned (lanes, window) per (op, limbs, ceil(log2 of the element count))
  std::mutex tune_mu;
  std::map<std::tuple<int, int, int>, std::pair<int, int>> tuned;
};

namespace pc2 {

// Scratch of at least `bytes` from the context (grows it outside stream capture).
uint32_t* ctx_scratch_get(pc2_ctx* ctx, size_t bytes);

// Key-owner encryption whose r-stream id is read on the device:
// (*round_ptr << 8) | kind (see EncCrtParams).
// `base`: position of element 0 of this call inside the tiled arrays.
int encrypt_round(pc2_ctx* ctx, const pc2_key* key, const uint64_t* d_m, size_t count, uint64_t seed,
                  const uint32_t* round_ptr, uint32_t kind, uint64_t e0, uint32_t* d_ct, cudaStream_t st,
                  size_t base = 0);
int hom_add_at(pc2_ctx* ctx, const pc2_key* key, const uint32_t* a, const uint32_t* b, size_t count, uint32_t* out,
               cudaStream_t st, size_t base);
int decrypt_at(pc2_ctx* ctx, const pc2_key* key, const uint32_t* ct, size_t count, uint32_t* out, cudaStream_t st,
               size_t base);

enum { OP_ENC_CRT = 0, OP_DEC = 1, OP_MATVEC = 2 };

// Lanes per element and window width (0 = key default) for `count` elements
// of operation `op` on `limbs`-limb operands: the context's forced lane count,
// else the autotuned entry for this size class, else the largest built lane
// count whose element groups still fit in one resident wave.
std::pair<int, int> pick_config(pc2_ctx* ctx, int op, int limbs, size_t count);
// Built lane counts for an operation and limb count (ascending).
const int* lane_set(int op, int limbs, int* n);

}  // namespace pc2
