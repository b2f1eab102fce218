#include "paillier_launch.cuh"

namespace pc2 {

template int launch_enc_pub<256, 4>(const EncPubParams<256>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t);
template int launch_hom_sum<256, 4>(const HomParams<256>&, size_t, uint32_t*, int, cudaStream_t, size_t);
template int launch_hom_scal<256, 4>(const HomParams<256>&, const uint32_t*, const uint64_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_hom_scal_wide<256, 4>(const HomParams<256>&, const uint32_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_enc_pub<256, 8>(const EncPubParams<256>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t);
template int launch_hom_sum<256, 8>(const HomParams<256>&, size_t, uint32_t*, int, cudaStream_t, size_t);
template int launch_hom_scal<256, 8>(const HomParams<256>&, const uint32_t*, const uint64_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_hom_scal_wide<256, 8>(const HomParams<256>&, const uint32_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);

}  // namespace pc2
