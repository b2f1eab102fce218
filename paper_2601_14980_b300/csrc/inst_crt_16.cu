#include "paillier_launch.cuh"

namespace pc2 {

template int launch_enc_crt<16, 1>(const EncCrtParams<16>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t, size_t);
template int launch_dec_crt<16, 1>(const DecParams<16>&, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t, size_t);
template int launch_enc_crt<16, 2>(const EncCrtParams<16>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t, size_t);
template int launch_dec_crt<16, 2>(const DecParams<16>&, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t, size_t);
template int launch_enc_crt<16, 4>(const EncCrtParams<16>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t, size_t);
template int launch_dec_crt<16, 4>(const DecParams<16>&, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t, size_t);
template int launch_enc_crt<16, 8>(const EncCrtParams<16>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t, size_t);
template int launch_dec_crt<16, 8>(const DecParams<16>&, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t, size_t);
template int launch_dec_crt_fixed<16, 1>(const DecParams<16>&, const uint32_t*, size_t, uint32_t*, uint32_t*, size_t, int, cudaStream_t);

template int launch_enc_crt2<16, 2>(const EncCrtParams<16>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t, size_t);
template int launch_dec_crt2<16, 2>(const DecParams<16>&, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t, size_t);
template int launch_enc_crt2<16, 4>(const EncCrtParams<16>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t, size_t);
template int launch_dec_crt2<16, 4>(const DecParams<16>&, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t, size_t);
template int launch_enc_crt2<16, 8>(const EncCrtParams<16>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t, size_t);
template int launch_dec_crt2<16, 8>(const DecParams<16>&, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t, size_t);

template int launch_enc_crt2<16, 1>(const EncCrtParams<16>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t, size_t);
template int launch_dec_crt2<16, 1>(const DecParams<16>&, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t, size_t);

}  // namespace pc2
