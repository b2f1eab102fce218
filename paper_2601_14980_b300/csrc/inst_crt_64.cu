#include "paillier_launch.cuh"

namespace pc2 {

template int launch_enc_crt<64, 1>(const EncCrtParams<64>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t, size_t);
template int launch_dec_crt<64, 1>(const DecParams<64>&, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t, size_t);
template int launch_enc_crt<64, 2>(const EncCrtParams<64>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t, size_t);
template int launch_dec_crt<64, 2>(const DecParams<64>&, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t, size_t);
template int launch_enc_crt<64, 4>(const EncCrtParams<64>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t, size_t);
template int launch_dec_crt<64, 4>(const DecParams<64>&, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t, size_t);
template int launch_enc_crt<64, 8>(const EncCrtParams<64>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t, size_t);
template int launch_dec_crt<64, 8>(const DecParams<64>&, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t, size_t);
template int launch_dec_crt_fixed<64, 1>(const DecParams<64>&, const uint32_t*, size_t, uint32_t*, uint32_t*, size_t, int, cudaStream_t);

template int launch_enc_crt2<64, 2>(const EncCrtParams<64>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t, size_t);
template int launch_dec_crt2<64, 2>(const DecParams<64>&, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t, size_t);
template int launch_enc_crt2<64, 4>(const EncCrtParams<64>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t, size_t);
template int launch_dec_crt2<64, 4>(const DecParams<64>&, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t, size_t);
template int launch_enc_crt2<64, 8>(const EncCrtParams<64>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t, size_t);
template int launch_dec_crt2<64, 8>(const DecParams<64>&, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t, size_t);

template int launch_enc_crt2<64, 1>(const EncCrtParams<64>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t, size_t);
template int launch_dec_crt2<64, 1>(const DecParams<64>&, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t, size_t);

}  // namespace pc2
