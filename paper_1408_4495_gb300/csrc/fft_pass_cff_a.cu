// Float-float FFT pass launchers for L = 16, 32, 48, 64, 96, 128, 256 (see fft_passes.cuh).
#include "fft_passes.cuh"

namespace ls {

LS_PASS_INST(, ffc, 16)
LS_PASS_INST(, ffc, 32)
LS_PASS_INST(, ffc, 48)
LS_PASS_INST(, ffc, 64)
LS_PASS_INST(, ffc, 96)
LS_PASS_INST(, ffc, 128)
LS_PASS_INST(, ffc, 256)

}  // namespace ls
