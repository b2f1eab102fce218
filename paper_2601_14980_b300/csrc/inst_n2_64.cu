#include "paillier_launch.cuh"

namespace pc2 {

template int launch_enc_pub<64, 1>(const EncPubParams<64>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t);
template int launch_hom_sum<64, 1>(const HomParams<64>&, size_t, uint32_t*, int, cudaStream_t, size_t);
template int launch_hom_scal<64, 1>(const HomParams<64>&, const uint32_t*, const uint64_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_hom_scal_wide<64, 1>(const HomParams<64>&, const uint32_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_enc_pub<64, 2>(const EncPubParams<64>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t);
template int launch_hom_sum<64, 2>(const HomParams<64>&, size_t, uint32_t*, int, cudaStream_t, size_t);
template int launch_hom_scal<64, 2>(const HomParams<64>&, const uint32_t*, const uint64_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_hom_scal_wide<64, 2>(const HomParams<64>&, const uint32_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_enc_pub<64, 4>(const EncPubParams<64>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t);
template int launch_hom_sum<64, 4>(const HomParams<64>&, size_t, uint32_t*, int, cudaStream_t, size_t);
template int launch_hom_scal<64, 4>(const HomParams<64>&, const uint32_t*, const uint64_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_hom_scal_wide<64, 4>(const HomParams<64>&, const uint32_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_enc_pub<64, 8>(const EncPubParams<64>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t);
template int launch_hom_sum<64, 8>(const HomParams<64>&, size_t, uint32_t*, int, cudaStream_t, size_t);
template int launch_hom_scal<64, 8>(const HomParams<64>&, const uint32_t*, const uint64_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_hom_scal_wide<64, 8>(const HomParams<64>&, const uint32_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);

}  // namespace pc2
