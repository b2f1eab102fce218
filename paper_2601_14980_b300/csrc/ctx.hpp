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
  int split = 0;          // CRT halves in parallel: 0 automatic, 1 never, 2 whenever lanes > 1
  int engine = -1;        // full-width powers at 2048-bit n: -1 automatic, 0 integer pipe, 1 tensor cores
  bool timing = false;    // record the stage boundaries of tensor-core calls
  cudaEvent_t ev[5] = {};  // before set-up, after set-up, after power mod p^2, after power mod q^2, after finish
  bool ev_recorded = false;
  // autotuned (lanes, window, split) per (op, limbs, ceil(log2 of the element count))
  std::mutex tune_mu;
  std::map<std::tuple<int, int, int>, std::tuple<int, int, int>> tuned;
};

namespace pc2 {

// Scratch of at least `bytes` from the context (grows it outside stream capture).
uint32_t* ctx_scratch_get(pc2_ctx* ctx, size_t bytes);

// Key-owner encryption whose r-stream id is read on the device:
// (*round_ptr << 8) | kind (see EncCrtParams).
// `base`: position of element 0 of this call inside the tiled arrays.
// Elements e >= split form a second vector (r-stream kind2, counter e0 + e - split,
// tiled position base2 + e - split): one launch when the split-halves kernel
// runs, two launches otherwise.
int encrypt_round(pc2_ctx* ctx, const pc2_key* key, const uint64_t* d_m, size_t count, uint64_t seed,
                  const uint32_t* round_ptr, uint32_t kind, uint64_t e0, uint32_t* d_ct, cudaStream_t st,
                  size_t base = 0, size_t split = ~(size_t)0, uint32_t kind2 = 0, size_t base2 = 0);
int hom_add_at(pc2_ctx* ctx, const pc2_key* key, const uint32_t* a, const uint32_t* b, size_t count, uint32_t* out,
               cudaStream_t st, size_t base);
int decrypt_at(pc2_ctx* ctx, const pc2_key* key, const uint32_t* ct, size_t count, uint32_t* out, cudaStream_t st,
               size_t base);

enum { OP_ENC_CRT = 0, OP_DEC = 1, OP_MATVEC = 2, OP_N2 = 3 };  // OP_N2: powers and products mod n^2

// Launch configuration of one call: lanes per element, window width (0 = key
// default) and whether the two CRT halves run in parallel (split, T > 1).
struct LaneCfg {
  int T;
  int w;
  bool split;
};
// For `count` elements of operation `op` on `limbs`-limb operands: the
// context's forced lane count, else the autotuned entry for this size class,
// else the most lanes per element (T, doubled when split) whose groups still
// fit in one resident wave, split preferred at equal lanes.
LaneCfg pick_config(pc2_ctx* ctx, int op, int limbs, size_t count);
// Built lane counts for an operation and limb count (ascending).
const int* lane_set(int op, int limbs, int* n);

}  // namespace pc2
