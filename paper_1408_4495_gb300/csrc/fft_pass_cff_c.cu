// Float-float FFT pass launchers for L = 2048, 4096 (see fft_passes.cuh).
#include "fft_passes.cuh"

namespace ls {

LS_PASS_INST(, ffc, 2048)
LS_PASS_INST(, ffc, 4096)

}  // namespace ls
