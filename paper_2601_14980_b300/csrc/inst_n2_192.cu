#include "paillier_launch.cuh"

namespace pc2 {

template int launch_enc_pub<192, 4>(const EncPubParams<192>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t);
template int launch_hom_sum<192, 4>(const HomParams<192>&, size_t, uint32_t*, int, cudaStream_t, size_t);
template int launch_hom_scal<192, 4>(const HomParams<192>&, const uint32_t*, const uint64_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_hom_scal_wide<192, 4>(const HomParams<192>&, const uint32_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_enc_pub<192, 8>(const EncPubParams<192>&, const uint64_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int*, int, cudaStream_t);
template int launch_hom_sum<192, 8>(const HomParams<192>&, size_t, uint32_t*, int, cudaStream_t, size_t);
template int launch_hom_scal<192, 8>(const HomParams<192>&, const uint32_t*, const uint64_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);
template int launch_hom_scal_wide<192, 8>(const HomParams<192>&, const uint32_t*, const uint32_t*, size_t, uint32_t*, ScratchFn, void*, int, cudaStream_t);

}  // namespace pc2
