// inst_mv_64.cu -- encrypted matvec kernels for 64-limb n^2.
#include "admm_kernels.cuh"

namespace pc2 {

template int launch_to_mont_rows<64, 1>(const ModConst<64>&, const uint32_t*, int, uint32_t*, int, cudaStream_t);
template size_t matvec_scratch_words<64, 1>(int, int);
template int launch_matvec<64, 1>(const MatvecParams<64>&, const uint32_t*, const uint32_t*, const uint32_t*,
                                   const long long*, const int*, const int*, const int*, uint32_t*, uint32_t*, int,
                                   cudaStream_t);
template int matvec_grid<64, 1>(int, int);
template int launch_to_mont_rows<64, 2>(const ModConst<64>&, const uint32_t*, int, uint32_t*, int, cudaStream_t);
template size_t matvec_scratch_words<64, 2>(int, int);
template int launch_matvec<64, 2>(const MatvecParams<64>&, const uint32_t*, const uint32_t*, const uint32_t*,
                                   const long long*, const int*, const int*, const int*, uint32_t*, uint32_t*, int,
                                   cudaStream_t);
template int matvec_grid<64, 2>(int, int);
template int launch_to_mont_rows<64, 4>(const ModConst<64>&, const uint32_t*, int, uint32_t*, int, cudaStream_t);
template size_t matvec_scratch_words<64, 4>(int, int);
template int launch_matvec<64, 4>(const MatvecParams<64>&, const uint32_t*, const uint32_t*, const uint32_t*,
                                   const long long*, const int*, const int*, const int*, uint32_t*, uint32_t*, int,
                                   cudaStream_t);
template int matvec_grid<64, 4>(int, int);
template int launch_to_mont_rows<64, 8>(const ModConst<64>&, const uint32_t*, int, uint32_t*, int, cudaStream_t);
template size_t matvec_scratch_words<64, 8>(int, int);
template int launch_matvec<64, 8>(const MatvecParams<64>&, const uint32_t*, const uint32_t*, const uint32_t*,
                                   const long long*, const int*, const int*, const int*, uint32_t*, uint32_t*, int,
                                   cudaStream_t);
template int matvec_grid<64, 8>(int, int);

template int launch_matvec_win<64, 1>(const MatvecParams<64>&, const uint32_t*, const uint32_t*, const uint32_t*,
                                      const long long*, const int*, const int*, const int*, int, uint32_t*, uint32_t*,
                                      uint32_t*, int, int, cudaStream_t);
template int matvec_win_grid<64, 1>(int, int);
template int launch_matvec_win<64, 2>(const MatvecParams<64>&, const uint32_t*, const uint32_t*, const uint32_t*,
                                      const long long*, const int*, const int*, const int*, int, uint32_t*, uint32_t*,
                                      uint32_t*, int, int, cudaStream_t);
template int matvec_win_grid<64, 2>(int, int);
template int launch_matvec_win<64, 4>(const MatvecParams<64>&, const uint32_t*, const uint32_t*, const uint32_t*,
                                      const long long*, const int*, const int*, const int*, int, uint32_t*, uint32_t*,
                                      uint32_t*, int, int, cudaStream_t);
template int matvec_win_grid<64, 4>(int, int);
template int launch_matvec_win<64, 8>(const MatvecParams<64>&, const uint32_t*, const uint32_t*, const uint32_t*,
                                      const long long*, const int*, const int*, const int*, int, uint32_t*, uint32_t*,
                                      uint32_t*, int, int, cudaStream_t);
template int matvec_win_grid<64, 8>(int, int);

}  // namespace pc2
