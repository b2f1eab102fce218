#include "paillier_launch.cuh"

namespace pc2 {

template int launch_enc_pub<16, 1>(const EncPubParams<16>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t);
template int launch_hom_sum<16, 1>(const HomParams<16>&, size_t, uint32_t*, int, cudaStream_t, size_t);
template int launch_hom_scal<16, 1>(const HomParams<16>&, const uint32_t*, const uint64_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_hom_scal_wide<16, 1>(const HomParams<16>&, const uint32_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_enc_pub<16, 2>(const EncPubParams<16>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t);
template int launch_hom_sum<16, 2>(const HomParams<16>&, size_t, uint32_t*, int, cudaStream_t, size_t);
template int launch_hom_scal<16, 2>(const HomParams<16>&, const uint32_t*, const uint64_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_hom_scal_wide<16, 2>(const HomParams<16>&, const uint32_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_enc_pub<16, 4>(const EncPubParams<16>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t);
template int launch_hom_sum<16, 4>(const HomParams<16>&, size_t, uint32_t*, int, cudaStream_t, size_t);
template int launch_hom_scal<16, 4>(const HomParams<16>&, const uint32_t*, const uint64_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_hom_scal_wide<16, 4>(const HomParams<16>&, const uint32_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);

}  // namespace pc2
