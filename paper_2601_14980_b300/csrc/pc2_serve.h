// pc2_serve.h -- internal structures of the serving form: a request loop
// that keeps the key and the requests' buffers on the device and runs the
// active requests' encrypt / decrypt / aggregate work together, one
// persistent launch per step, with new requests joining at the next step.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "pc2_params.h"

namespace pc2 {

enum { SERVE_ENCRYPT = 1, SERVE_DECRYPT = 2, SERVE_AGGREGATE = 3 };
// Work-item kinds: the operation and the lanes per element (1: one lane;
// 2, 8: that many lanes per CRT half, the two halves in parallel).
enum { SK_ENC1 = 0, SK_ENC8 = 1, SK_DEC1 = 2, SK_DEC8 = 3, SK_AGG = 4, SK_ENC2 = 5, SK_DEC2 = 6, SK_ENC1S = 7,
       SK_DEC1S = 8 };  // *1S: one lane per CRT half, halves in parallel
constexpr int kServeLanesSmall = 8;  // lanes per CRT half for small requests (halves in parallel: lower latency)

// Lanes per element of an aggregation item: 32 limbs per lane.
constexpr int serve_agg_lanes(int L2) { return L2 >= 64 ? L2 / 32 : 1; }

// A request as one step's kernel sees it (device table, one entry per active request).
struct ServeReq {
  const uint64_t* m64;    // encrypt: plaintexts (uint64)
  const uint32_t* ct_in;  // decrypt: tiled ciphertexts; aggregate: `groups` tiled arrays, ct_stride words apart
  uint32_t* out;          // tiled ciphertexts (encrypt, aggregate) or plaintexts (decrypt)
  uint64_t count;
  uint64_t ct_stride;
  uint64_t seed;          // encrypt: Philox key, r-stream and counter base as pc2_encrypt
  uint64_t e0;
  uint32_t stream;
  uint32_t op;
  uint32_t groups;
  uint32_t pad_;
};

struct ServeItem {
  uint32_t req;    // index into the step's request table
  uint32_t first;  // first element
  uint32_t count;  // elements (<= 128 / lanes)
  uint32_t kind;   // SK_*
};

// Key constants in device memory (one key per server).
template <int Lh>
struct ServeKey {
  EncCrtParams<Lh> enc;
  DecParams<Lh> dec;
  ModConst<2 * Lh> n2;
  uint32_t rpow[kMaxGroups + 1][2 * Lh];  // R^g mod n^2, g = 0..kMaxGroups (fix-up of a g-operand product)
};

// The moduli read with compile-time offsets by one-lane products, in constant memory.
template <int Lh>
struct ServeConst {
  uint32_t mp[Lh];      // p^2
  uint32_t mq[Lh];      // q^2
  uint32_t n2[2 * Lh];  // n^2
  uint32_t hp[Lh / 2];  // p
  uint32_t hq[Lh / 2];  // q
};

struct ServeParams {
  const void* key;          // ServeKey<Lh>*
  const ServeReq* reqs;
  const ServeItem* items;
  uint32_t nitems;
  int tabw;                 // words per group of the window table
  uint32_t* next;           // next unclaimed item (zeroed before the launch)
  uint32_t* scratch;
  size_t cta_words;
  int* status;
};

// one_lane_split: run the SK_ENC1S / SK_DEC1S items (k_serve_step_s1) instead of the others.
template <int Lh>
int launch_serve_step(const ServeParams& P, size_t smem, int grid, cudaStream_t st, bool one_lane_split);
// Copies a key's one-lane moduli to constant memory (synchronises `st`); the
// constant block is shared by every server of this key size in the process.
template <int Lh>
int serve_set_const(const ServeConst<Lh>* d_const, cudaStream_t st);
template <int Lh>
int serve_blocks_per_sm(size_t smem);

}  // namespace pc2
