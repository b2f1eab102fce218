#include "paillier_launch.cuh"

namespace pc2 {

template int launch_enc_crt<128, 2>(const EncCrtParams<128>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t, size_t);
template int launch_dec_crt<128, 2>(const DecParams<128>&, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t, size_t);
template int launch_enc_crt<128, 4>(const EncCrtParams<128>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t, size_t);
template int launch_dec_crt<128, 4>(const DecParams<128>&, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t, size_t);
template int launch_enc_crt<128, 8>(const EncCrtParams<128>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t, size_t);
template int launch_dec_crt<128, 8>(const DecParams<128>&, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t, size_t);

template int launch_enc_crt2<128, 2>(const EncCrtParams<128>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t, size_t);
template int launch_dec_crt2<128, 2>(const DecParams<128>&, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t, size_t);
template int launch_enc_crt2<128, 4>(const EncCrtParams<128>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t, size_t);
template int launch_dec_crt2<128, 4>(const DecParams<128>&, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t, size_t);
template int launch_enc_crt2<128, 8>(const EncCrtParams<128>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t, size_t);
template int launch_dec_crt2<128, 8>(const DecParams<128>&, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t, size_t);

}  // namespace pc2
