// inst_mv_32.cu -- encrypted matvec kernels for 32-limb n^2.
#include "admm_kernels.cuh"

namespace pc2 {

template int launch_to_mont_rows<32, 1>(const ModConst<32>&, const uint32_t*, int, uint32_t*, int, cudaStream_t);
template size_t matvec_scratch_words<32, 1>(int, int);
template int launch_matvec<32, 1>(const MatvecParams<32>&, const uint32_t*, const uint32_t*, const uint32_t*,
                                   const long long*, const int*, const int*, const int*, uint32_t*, uint32_t*, int,
                                   cudaStream_t);
template int matvec_grid<32, 1>(int, int);
template int launch_to_mont_rows<32, 2>(const ModConst<32>&, const uint32_t*, int, uint32_t*, int, cudaStream_t);
template size_t matvec_scratch_words<32, 2>(int, int);
template int launch_matvec<32, 2>(const MatvecParams<32>&, const uint32_t*, const uint32_t*, const uint32_t*,
                                   const long long*, const int*, const int*, const int*, uint32_t*, uint32_t*, int,
                                   cudaStream_t);
template int matvec_grid<32, 2>(int, int);
template int launch_to_mont_rows<32, 4>(const ModConst<32>&, const uint32_t*, int, uint32_t*, int, cudaStream_t);
template size_t matvec_scratch_words<32, 4>(int, int);
template int launch_matvec<32, 4>(const MatvecParams<32>&, const uint32_t*, const uint32_t*, const uint32_t*,
                                   const long long*, const int*, const int*, const int*, uint32_t*, uint32_t*, int,
                                   cudaStream_t);
template int matvec_grid<32, 4>(int, int);
template int launch_to_mont_rows<32, 8>(const ModConst<32>&, const uint32_t*, int, uint32_t*, int, cudaStream_t);
template size_t matvec_scratch_words<32, 8>(int, int);
template int launch_matvec<32, 8>(const MatvecParams<32>&, const uint32_t*, const uint32_t*, const uint32_t*,
                                   const long long*, const int*, const int*, const int*, uint32_t*, uint32_t*, int,
                                   cudaStream_t);
template int matvec_grid<32, 8>(int, int);

template int launch_matvec_win<32, 1>(const MatvecParams<32>&, const uint32_t*, const uint32_t*, const uint32_t*,
                                      const long long*, const int*, const int*, const int*, int, uint32_t*, uint32_t*,
                                      uint32_t*, int, int, cudaStream_t);
template int matvec_win_grid<32, 1>(int, int);
template int launch_matvec_win<32, 2>(const MatvecParams<32>&, const uint32_t*, const uint32_t*, const uint32_t*,
                                      const long long*, const int*, const int*, const int*, int, uint32_t*, uint32_t*,
                                      uint32_t*, int, int, cudaStream_t);
template int matvec_win_grid<32, 2>(int, int);
template int launch_matvec_win<32, 4>(const MatvecParams<32>&, const uint32_t*, const uint32_t*, const uint32_t*,
                                      const long long*, const int*, const int*, const int*, int, uint32_t*, uint32_t*,
                                      uint32_t*, int, int, cudaStream_t);
template int matvec_win_grid<32, 4>(int, int);
template int launch_matvec_win<32, 8>(const MatvecParams<32>&, const uint32_t*, const uint32_t*, const uint32_t*,
                                      const long long*, const int*, const int*, const int*, int, uint32_t*, uint32_t*,
                                      uint32_t*, int, int, cudaStream_t);
template int matvec_win_grid<32, 8>(int, int);

}  // namespace pc2
