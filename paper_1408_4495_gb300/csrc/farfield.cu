// Far-field pattern of the scattered field (exterior evaluation after the solve).
//
// The total field u = u_I + u_s solves u + K(omega^2 m u) = u_I (Sec. 1, eq. ls), so outside
// the domain u_s(x) = -int G(x - y) omega^2 m(y) u(y) dy.  With the large-|x| form of the
// Green's function, G(x - y) ~ c_d e^{i omega r} r^{-(d-1)/2} e^{-i omega theta . y} in the
// direction theta = x / r, the scattered field behaves as e^{i omega r} r^{-(d-1)/2} u_inf:
//   u_inf(theta) = -c_d h^d sum_i e^{-i omega theta . x_i} w_i (u_I(x_i) + u_s,i),
//   w = omega^2 m,  c_2 = e^{i pi/4} / sqrt(8 pi omega),  c_3 = 1 / (4 pi),
// the integral replaced by the Nystrom quadrature of K.  Both exponentials factor over the
// axes, so each block tabulates e^{-i omega theta_a x} and e^{i omega (d_a - theta_a) x} per
// axis in shared memory (FP64) and a grid point costs d - 1 complex products per factor.
#include <atomic>
#include <cmath>

#include "common.cuh"
#include "kernels.h"
#include "prof.h"

namespace ls {

// grid (observation directions, right-hand sides); dynamic shared memory: 2 d n double2
__global__ void __launch_bounds__(256) k_far_field(int d, int n, int nobs, const double2* __restrict__ us,
                                                   const double* __restrict__ dirs, const double* __restrict__ obs,
                                                   const double* __restrict__ w, double omega, double h, double2 cd,
                                                   double2* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* te = reinterpret_cast<double2*>(smem_raw);  // [d][n] e^{-i omega theta_a x_j}
  double2* ti = te + (size_t)d * n;                     // [d][n] e^{i omega (d_a - theta_a) x_j}
  __shared__ double2 red[256 / 32];
  const int k = blockIdx.x, r = blockIdx.y;
  const double* th = obs + (size_t)k * d;
  const double* di = dirs + (size_t)r * d;
  for (int e = threadIdx.x; e < d * n; e += blockDim.x) {
    const int a = e / n, j = e - a * n;
    const double x = (j + 1) * h;
    double s1, c1, s2, c2;
    sincos(-omega * th[a] * x, &s1, &c1);
    sincos(omega * (di[a] - th[a]) * x, &s2, &c2);
    te[e] = make_double2(c1, s1);
    ti[e] = make_double2(c2, s2);
  }
  __syncthreads();
  const long N = d == 2 ? (long)n * n : (long)n * n * n;
  const double2* u = us + (size_t)r * N;
  double2 acc = make_double2(0.0, 0.0);
  for (long i = threadIdx.x; i < N; i += blockDim.x) {
    const double wi = w[i];
    if (wi == 0.0) continue;
    long q = i;
    double2 fe = make_double2(1.0, 0.0), fi = make_double2(1.0, 0.0);
    for (int a = d - 1; a >= 0; --a) {
      const int j = (int)(q % n);
      q /= n;
      fe = cmul(fe, te[(size_t)a * n + j]);
      fi = cmul(fi, ti[(size_t)a * n + j]);
    }
    // e^{-i omega theta.x} w (u_I + u_s) = w (e^{i omega (d - theta).x} + e^{-i omega theta.x} u_s)
    const double2 v = cadd(fi, cmul(fe, u[i]));
    acc.x = fma(wi, v.x, acc.x);
    acc.y = fma(wi, v.y, acc.y);
  }
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 s = make_double2(0.0, 0.0);
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s = cadd(s, red[q]);
    const double hd = d == 2 ? h * h : h * h * h;
    const double2 v = cmul(cd, s);
    out[(size_t)r * nobs + k] = make_double2(-hd * v.x, -hd * v.y);
  }
}

void far_field(int d, int n, int nrhs, int nobs, const double2* us, const double* dirs, const double* obs,
               const double* w, double omega, double h, double2* out, cudaStream_t st) {
  const double2 cd = d == 2 ? make_double2(cos(M_PI / 4) / sqrt(8 * M_PI * omega), sin(M_PI / 4) / sqrt(8 * M_PI * omega))
                            : make_double2(1.0 / (4 * M_PI), 0.0);
  const size_t smem = 2 * (size_t)d * n * sizeof(double2);
  static std::atomic<bool> attr{false};  // set once per process; repeats are harmless
  if (!attr.load(std::memory_order_acquire)) {
    LS_CUDA(cudaFuncSetAttribute(k_far_field, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 2 * 2048 * 16));
    attr.store(true, std::memory_order_release);
  }
  LS_LAUNCH("far_field", st,
            k_far_field<<<dim3(nobs, nrhs), 256, smem, st>>>(d, n, nobs, us, dirs, obs, w, omega, h, cd, out));
}

}  // namespace ls
