// The FFT passes in FP64 arithmetic (see fft_passes.cuh).
#include "fft_passes.cuh"

namespace ls {

template void row_pass<double2>(int, int, const RowPassArgs&, cudaStream_t);
template void col_pass<double2>(int, int, const ColPassArgs&, cudaStream_t);

}  // namespace ls
