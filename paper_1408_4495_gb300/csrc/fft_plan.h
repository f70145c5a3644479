// Radix plan of the Stockham line transforms and the layout of the FP32 passes' twiddle
// table, shared by the passes (device) and the table's construction (host).
//
// A line of length L (2^k or 3 * 2^k) is transformed by passes of radix 8 while the remaining
// length is a multiple of 8, then 4 or 2, then 3.  The pass that starts from sub-transforms
// of length NS (NS > 1) multiplies entry r of butterfly k (0 <= k < NS, 0 <= r < R) by
// w^{r k}, w = exp(-2 pi i / (NS R)) (conjugated in the inverse transform).  The FP32 table
// holds these factors pass after pass, butterfly after butterfly: pass NS at
// tw_pass_offset(L, NS), butterfly k's R factors (r = 0 included) at k * R from there, so
// that a butterfly reads one contiguous, 16-byte aligned run (sum over the passes of NS * R
// < 2 L entries).  The FP64 and float-float passes index the L-entry table exp(-2 pi i m / L)
// at m = r k L / (NS R) instead: with 16-byte entries the per-butterfly runs spread one load
// instruction of a warp over more cache lines than that table's neighbouring entries do.
#pragma once

#if defined(__CUDACC__)
#define LS_FFT_HD __host__ __device__
#else
#define LS_FFT_HD
#endif

namespace ls {

LS_FFT_HD constexpr int pass_radix(int L, int NS) {
  return (L / NS) % 8 == 0 ? 8 : ((L / NS) % 4 == 0 ? 4 : ((L / NS) % 2 == 0 ? 2 : 3));
}
LS_FFT_HD constexpr int last_radix(int L) {
  int NS = 1;
  while (NS * pass_radix(L, NS) < L) NS *= pass_radix(L, NS);
  return pass_radix(L, NS);
}
// first entry of the factors of the pass that starts from length NS (NS > 1)
LS_FFT_HD constexpr int tw_pass_offset(int L, int NS) {
  int off = 0, ns = 1;
  while (ns < NS) {
    const int R = pass_radix(L, ns);
    if (ns > 1) off += ns * R;
    ns *= R;
  }
  return off;
}
// entries of the whole table
LS_FFT_HD constexpr int tw_table_size(int L) { return tw_pass_offset(L, L); }

}  // namespace ls
