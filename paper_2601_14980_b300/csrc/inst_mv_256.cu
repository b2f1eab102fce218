// inst_mv_256.cu -- encrypted matvec kernels for 256-limb n^2.
#include "admm_kernels.cuh"

namespace pc2 {

template int launch_to_mont_rows<256, 4>(const ModConst<256>&, const uint32_t*, int, uint32_t*, int, cudaStream_t);
template size_t matvec_scratch_words<256, 4>(int, int);
template int launch_matvec<256, 4>(const MatvecParams<256>&, const uint32_t*, const uint32_t*, const uint32_t*,
                                   const long long*, const int*, const int*, const int*, uint32_t*, uint32_t*, int,
                                   cudaStream_t);
template int matvec_grid<256, 4>(int, int);
template int launch_to_mont_rows<256, 8>(const ModConst<256>&, const uint32_t*, int, uint32_t*, int, cudaStream_t);
template size_t matvec_scratch_words<256, 8>(int, int);
template int launch_matvec<256, 8>(const MatvecParams<256>&, const uint32_t*, const uint32_t*, const uint32_t*,
                                   const long long*, const int*, const int*, const int*, uint32_t*, uint32_t*, int,
                                   cudaStream_t);
template int matvec_grid<256, 8>(int, int);

template int launch_matvec_win<256, 4>(const MatvecParams<256>&, const uint32_t*, const uint32_t*, const uint32_t*,
                                      const long long*, const int*, const int*, const int*, int, uint32_t*, uint32_t*,
                                      uint32_t*, int, int, cudaStream_t);
template int matvec_win_grid<256, 4>(int, int);
template int launch_matvec_win<256, 8>(const MatvecParams<256>&, const uint32_t*, const uint32_t*, const uint32_t*,
                                      const long long*, const int*, const int*, const int*, int, uint32_t*, uint32_t*,
                                      uint32_t*, int, int, cudaStream_t);
template int matvec_win_grid<256, 8>(int, int);

}  // namespace pc2
