// Weight k_0 of the singular point of the Nystrom table (Sec. 2.1), on the host in FP64.
//
// rule 0: the integral of G over the disk (2D) / ball (3D) of area / volume h^d centred at
//   the origin, in closed form (2D: (i pi a / 2 omega) H_1(omega a) - 1/omega^2, a = h/sqrt(pi);
//   3D: e^{i omega a}(1/omega^2 - i a/omega) - 1/omega^2, a = h (3/(4 pi))^{1/3}; 3D Laplace
//   (omega = 0): a^2 / 2).  Second-order accurate.
// rule 1: the one-point correction of the trapezoidal rule (Sec. 2.1 states O(h^4 log 1/h)):
//   the weight for which sum_{j != 0} G(h j) h^d f(h j) + k_0 f(0) integrates G f exactly for
//   the Gaussian f = exp(-|x|^2 / (2 s^2)), s = 8 h.  The plain trapezoidal error is f(0)
//   times a constant plus O(h^4 log h) terms, so one smooth f fixes the weight to that order.
//   The lattice sum runs over |j_a| <= 88 (11 s / h); the radial integral of G f over
//   [0, 12 s] uses Gauss-Legendre panels, graded geometrically towards r = 0 where the 2D
//   integrand has its r log r behaviour.
#include <cmath>
#include <complex>
#include <vector>

#include "ls.h"

namespace {

using cd = std::complex<double>;

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on P_n from the Chebyshev
// guesses, the recurrence for P_n and its derivative)
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// G(r) for r > 0: 2D (i/4) H_0^(1)(omega r), 3D e^{i omega r} / (4 pi r)
cd green(int d, double omega, double r) {
  if (d == 2) return cd(-0.25 * std::cyl_neumann(0.0, omega * r), 0.25 * std::cyl_bessel_j(0.0, omega * r));
  return std::exp(cd(0.0, omega * r)) / (4.0 * M_PI * r);
}

cd k0_ball(int d, double omega, double h) {
  if (d == 2) {
    const double a = h / std::sqrt(M_PI), z = omega * a, f = M_PI * a / (2.0 * omega);
    return cd(-f * std::cyl_neumann(1.0, z) - 1.0 / (omega * omega), f * std::cyl_bessel_j(1.0, z));
  }
  const double a = h * std::cbrt(3.0 / (4.0 * M_PI));
  if (omega == 0.0) return cd(0.5 * a * a, 0.0);
  const cd e = std::exp(cd(0.0, omega * a));
  return e * cd(1.0 / (omega * omega), -a / omega) - cd(1.0 / (omega * omega), 0.0);
}

// Neumaier's compensated summation (improved Kahan-Babuska), on each of re and im: the
// lattice sum adds ~10^6 terms and k_0 is the small difference of it and the integral, so
// plain accumulation loses ~1e-10 of k_0
struct SumC {
  double s[2] = {0.0, 0.0}, c[2] = {0.0, 0.0};
  void add(cd v) {
    const double x[2] = {v.real(), v.imag()};
    for (int p = 0; p < 2; ++p) {
      const double t = s[p] + x[p];
      c[p] += std::fabs(s[p]) >= std::fabs(x[p]) ? (s[p] - t) + x[p] : (x[p] - t) + s[p];
      s[p] = t;
    }
  }
  cd value() const { return cd(s[0] + c[0], s[1] + c[1]); }
};

cd k0_corrected(int d, double omega, double h) {
  const double s = 8.0 * h;
  const int M = 88;
  // lattice sum over j != 0 (by symmetry over the nonnegative octant with multiplicities)
  SumC lat;
  const double hd = d == 2 ? h * h : h * h * h;
  const int kmax = d == 2 ? 0 : M;
  for (int i = 0; i <= M; ++i)
    for (int j = 0; j <= M; ++j)
      for (int k = 0; k <= kmax; ++k) {
        if (i == 0 && j == 0 && k == 0) continue;
        const double mult = (i ? 2.0 : 1.0) * (j ? 2.0 : 1.0) * (d == 3 && k ? 2.0 : 1.0);
        const double r = h * std::sqrt((double)i * i + (double)j * j + (double)k * k);
        lat.add(mult * green(d, omega, r) * hd * std::exp(-r * r / (2.0 * s * s)));
      }
  // radial integral of G f over [0, 12 s]
  auto g = [&](double r) -> cd {
    const double wgt = std::exp(-r * r / (2.0 * s * s));
    if (d == 2) return 2.0 * M_PI * r * green(2, omega, r) * wgt;
    return r * std::exp(cd(0.0, omega * r)) * wgt;  // 4 pi r^2 e^{i omega r} / (4 pi r)
  };
  std::vector<double> gx, gw;
  gauss_legendre(48, gx, gw);
  auto panel = [&](double a, double b) {
    cd acc = 0.0;
    for (size_t q = 0; q < gx.size(); ++q) acc += gw[q] * g(0.5 * (b - a) * gx[q] + 0.5 * (a + b));
    return 0.5 * (b - a) * acc;
  };
  const double R = 12.0 * s, first = R / 64.0;
  cd integral = 0.0;
  for (int p = 1; p < 64; ++p) integral += panel(first * p, first * (p + 1));
  double hi = first;
  for (int lev = 0; lev < 40; ++lev) {  // [first / 2^(lev+1), first / 2^lev]
    integral += panel(0.5 * hi, hi);
    hi *= 0.5;
  }
  return integral - lat.value();
}

}  // namespace

extern "C" ls_status ls_k0_weight(int dim, double omega, double h, int rule, double* out) {
  if (!out || (dim != 2 && dim != 3) || !(h > 0) || !std::isfinite(omega) || omega < 0) return LS_EINVAL;
  if (dim == 2 && omega == 0.0) return LS_EINVAL;  // the Laplace variant is 3D (Sec. 5)
  if (rule != LS_K0_BALL && rule != LS_K0_CORRECTED) return LS_EINVAL;
  const cd k = rule == LS_K0_BALL ? k0_ball(dim, omega, h) : k0_corrected(dim, omega, h);
  out[0] = k.real();
  out[1] = k.imag();
  return LS_OK;
}
