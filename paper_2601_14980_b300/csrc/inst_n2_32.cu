#include "paillier_launch.cuh"

namespace pc2 {

template int launch_enc_pub<32, 1>(const EncPubParams<32>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t);
template int launch_hom_sum<32, 1>(const HomParams<32>&, size_t, uint32_t*, int, cudaStream_t, size_t);
template int launch_hom_scal<32, 1>(const HomParams<32>&, const uint32_t*, const uint64_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_hom_scal_wide<32, 1>(const HomParams<32>&, const uint32_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_enc_pub<32, 2>(const EncPubParams<32>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t);
template int launch_hom_sum<32, 2>(const HomParams<32>&, size_t, uint32_t*, int, cudaStream_t, size_t);
template int launch_hom_scal<32, 2>(const HomParams<32>&, const uint32_t*, const uint64_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_hom_scal_wide<32, 2>(const HomParams<32>&, const uint32_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_enc_pub<32, 4>(const EncPubParams<32>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t);
template int launch_hom_sum<32, 4>(const HomParams<32>&, size_t, uint32_t*, int, cudaStream_t, size_t);
template int launch_hom_scal<32, 4>(const HomParams<32>&, const uint32_t*, const uint64_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_hom_scal_wide<32, 4>(const HomParams<32>&, const uint32_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_enc_pub<32, 8>(const EncPubParams<32>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t);
template int launch_hom_sum<32, 8>(const HomParams<32>&, size_t, uint32_t*, int, cudaStream_t, size_t);
template int launch_hom_scal<32, 8>(const HomParams<32>&, const uint32_t*, const uint64_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_hom_scal_wide<32, 8>(const HomParams<32>&, const uint32_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);

}  // namespace pc2
