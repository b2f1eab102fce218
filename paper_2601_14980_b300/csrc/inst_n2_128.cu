#include "paillier_launch.cuh"

namespace pc2 {

template int launch_enc_pub<128, 4>(const EncPubParams<128>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t);
template int launch_hom_sum<128, 4>(const HomParams<128>&, size_t, uint32_t*, int, cudaStream_t, size_t);
template int launch_hom_scal<128, 4>(const HomParams<128>&, const uint32_t*, const uint64_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_hom_scal_wide<128, 4>(const HomParams<128>&, const uint32_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_enc_pub<128, 8>(const EncPubParams<128>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t);
template int launch_hom_sum<128, 8>(const HomParams<128>&, size_t, uint32_t*, int, cudaStream_t, size_t);
template int launch_hom_scal<128, 8>(const HomParams<128>&, const uint32_t*, const uint64_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_hom_scal_wide<128, 8>(const HomParams<128>&, const uint32_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);

}  // namespace pc2
