// noalloc.cu -- decryption that allocates no device memory.
//
// pc2_decrypt (capi.cpp) takes its scratch from a pc2_ctx, which grows it with
// cudaMalloc on first use -- and growing also synchronises the device and
// frees the old buffer.  Some callers cannot do that: code running under a
// host memory/allocation policy that forbids new device allocations (a
// serving process with a fixed, pre-carved memory budget, or a plugin that
// must not touch the device allocator), or code on a latency path that cannot
// afford the device-wide synchronisation a cudaMalloc/cudaFree may imply.
// For them pc2_decrypt_noalloc runs the same decryption kernel with its
// scratch in a fixed array compiled into the library.
//
// The array below lives in device memory (a file-scope __device__ array, one
// copy per GPU that loads the library).  In host code its name is only a
// handle, not a device address: host code looks the address up once per
// device with cudaGetSymbolAddress and passes that address to the kernel.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/pc2.h"
#include "keys.hpp"
#include "pc2_kernels.h"

namespace {

constexpr size_t kNoAllocBytes = (size_t)PC2_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// Held by every GPU that loads the library, until the process exits.
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocBytes / sizeof(uint32_t)];

std::mutex g_mu;
uint32_t* g_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up on
// the first call for that device and cached for the life of the process; a
// cudaDeviceReset invalidates it, so the entry point must not be used across
// one).
int scratch_address(int dev, uint32_t** out) {
  if (dev < 0 || dev >= kMaxDevices) return PC2_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return PC2_ECUDA;
    g_addr[dev] = static_cast<uint32_t*>(p);
  }
  *out = g_addr[dev];
  return PC2_OK;
}

template <int Lh>
int dec_fixed(const pc2_key* key, const uint32_t* ct, size_t count, uint32_t* out, uint32_t* scratch, int sms,
              cudaStream_t st) {
  int rc = PC2_OK;
  auto P = pc2::dec_params<Lh>(key, &rc);
  if (!P) return rc;
  return pc2::launch_dec_crt_fixed<Lh, pc2::lanes_for(Lh)>(*P, ct, count, out, scratch,
                                                          kNoAllocBytes / sizeof(uint32_t), sms, st);
}

}  // namespace

extern "C" int pc2_decrypt_noalloc(const pc2_key* key, const uint32_t* d_ct, size_t count, uint32_t* d_m,
                                   pc2_stream_t stream) {
  if (!key) return PC2_EINVAL;
  if (!key->priv) return PC2_EKEY;
  if (!count) return PC2_OK;
  if (!d_ct || !d_m) return PC2_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PC2_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PC2_ECUDA;
  uint32_t* scratch = nullptr;
  int rc = scratch_address(dev, &scratch);
  if (rc != PC2_OK) return rc;
  const cudaStream_t st = (cudaStream_t)stream;
  switch (key->Lh) {
    case 8: return dec_fixed<8>(key, d_ct, count, d_m, scratch, sms, st);
    case 16: return dec_fixed<16>(key, d_ct, count, d_m, scratch, sms, st);
    case 32: return dec_fixed<32>(key, d_ct, count, d_m, scratch, sms, st);
    case 64: return dec_fixed<64>(key, d_ct, count, d_m, scratch, sms, st);
    case 96: return dec_fixed<96>(key, d_ct, count, d_m, scratch, sms, st);
    default: return PC2_EUNSUPPORTED;
  }
}
