// inst_mv_16.cu -- encrypted matvec kernels for 16-limb n^2.
#include "admm_kernels.cuh"

namespace pc2 {

template int launch_to_mont_rows<16, 1>(const ModConst<16>&, const uint32_t*, int, uint32_t*, int, cudaStream_t);
template size_t matvec_scratch_words<16, 1>(int, int);
template int launch_matvec<16, 1>(const MatvecParams<16>&, const uint32_t*, const uint32_t*, const uint32_t*,
                                   const long long*, const int*, const int*, const int*, uint32_t*, uint32_t*, int,
                                   cudaStream_t);
template int matvec_grid<16, 1>(int, int);
template int launch_to_mont_rows<16, 2>(const ModConst<16>&, const uint32_t*, int, uint32_t*, int, cudaStream_t);
template size_t matvec_scratch_words<16, 2>(int, int);
template int launch_matvec<16, 2>(const MatvecParams<16>&, const uint32_t*, const uint32_t*, const uint32_t*,
                                   const long long*, const int*, const int*, const int*, uint32_t*, uint32_t*, int,
                                   cudaStream_t);
template int matvec_grid<16, 2>(int, int);
template int launch_to_mont_rows<16, 4>(const ModConst<16>&, const uint32_t*, int, uint32_t*, int, cudaStream_t);
template size_t matvec_scratch_words<16, 4>(int, int);
template int launch_matvec<16, 4>(const MatvecParams<16>&, const uint32_t*, const uint32_t*, const uint32_t*,
                                   const long long*, const int*, const int*, const int*, uint32_t*, uint32_t*, int,
                                   cudaStream_t);
template int matvec_grid<16, 4>(int, int);

template int launch_matvec_win<16, 1>(const MatvecParams<16>&, const uint32_t*, const uint32_t*, const uint32_t*,
                                      const long long*, const int*, const int*, const int*, int, uint32_t*, uint32_t*,
                                      uint32_t*, int, int, cudaStream_t);
template int matvec_win_grid<16, 1>(int, int);
template int launch_matvec_win<16, 2>(const MatvecParams<16>&, const uint32_t*, const uint32_t*, const uint32_t*,
                                      const long long*, const int*, const int*, const int*, int, uint32_t*, uint32_t*,
                                      uint32_t*, int, int, cudaStream_t);
template int matvec_win_grid<16, 2>(int, int);
template int launch_matvec_win<16, 4>(const MatvecParams<16>&, const uint32_t*, const uint32_t*, const uint32_t*,
                                      const long long*, const int*, const int*, const int*, int, uint32_t*, uint32_t*,
                                      uint32_t*, int, int, cudaStream_t);
template int matvec_win_grid<16, 4>(int, int);

}  // namespace pc2
