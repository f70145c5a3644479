// The FFT passes in float-float arithmetic (see fft_passes.cuh): the dispatch over lengths;
// the launchers of each length are instantiated in fft_pass_cff_{a,b,c}.cu.
#include "fft_passes.cuh"

namespace ls {

#define LS_DECL(LL) LS_PASS_INST(extern, ffc, LL)
LS_FOR_L(LS_DECL)
#undef LS_DECL

template void row_pass<ffc>(int, int, const RowPassArgs&, cudaStream_t);
template void col_pass<ffc>(int, int, const ColPassArgs&, cudaStream_t);

}  // namespace ls
