// Float-float FFT pass launchers for L = 512, 1024 (see fft_passes.cuh).
#include "fft_passes.cuh"

namespace ls {

LS_PASS_INST(, ffc, 512)
LS_PASS_INST(, ffc, 1024)

}  // namespace ls
