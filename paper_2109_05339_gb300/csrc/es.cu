// Host-side set-up of the exponential-of-semicircle (ES) NUFFT kernel.
//
// The paper slices and merges with the FINUFFT / cuFINUFFT libraries
// (Sec. III-A), whose published method spreads with
//   phi(z) = exp(beta (sqrt(1 - z^2) - 1)),  |z| <= 1,
// over w fine-grid cells, w = ceil(log10(1/eps)) + 1, beta = 2.30 w, on a
// grid upsampled by 2. Deconvolution divides mode k by the kernel's Fourier
// transform; per axis the factor is
//   p_k = 2 / (w int_{-1}^{1} phi(z) cos(k a z) dz),  a = w pi / n_f,
// evaluated here in FP64 by Gauss-Legendre quadrature (nodes from Newton's
// method on the Legendre recurrence) and cast to float for the kernels.
#include <cmath>
#include <vector>

#include "plan.h"

namespace spf {

void es_params(double eps, int* w, double* beta) {
  *w = (int)std::ceil(std::log10(1.0 / eps)) + 1;
  *beta = 2.30 * (*w);
}

int smooth_even_at_least(int n) {
  if (n < 2) n = 2;
  if (n % 2) ++n;
  for (;; n += 2) {
    int m = n;
    while (m % 2 == 0) m /= 2;
    while (m % 3 == 0) m /= 3;
    while (m % 5 == 0) m /= 5;
    if (m == 1) return n;
  }
}

int fine_size(int n_modes, int w) { return smooth_even_at_least(std::max(2 * n_modes, 2 * w)); }

// Gauss-Legendre nodes and weights on [-1, 1].
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& wt) {
  x.assign(n, 0.0);
  wt.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      // P_n(z) and P_n'(z) by the three-term recurrence
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double pn = (n == 0) ? 1.0 : p1;
      double pm1 = (n == 1) ? 1.0 : p0;
      dp = n * (z * pn - pm1) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    double wi = 2.0 / ((1.0 - z * z) * dp * dp);
    wt[i] = wi;
    wt[n - 1 - i] = wi;
  }
}

void deconv_factors(int n_modes, int nf, int w, double beta, double* out) {
  const int nq = 256;
  std::vector<double> z, wq;
  gauss_legendre(nq, z, wq);
  std::vector<double> f(nq);
  for (int q = 0; q < nq; ++q) {
    double s = 1.0 - z[q] * z[q];
    f[q] = wq[q] * std::exp(beta * (std::sqrt(s > 0 ? s : 0) - 1.0));
  }
  const int Mh = (n_modes - 1) / 2;
  const double a = w * M_PI / nf;
  for (int k = -Mh; k <= Mh; ++k) {
    double J = 0.0;
    for (int q = 0; q < nq; ++q) J += f[q] * std::cos(k * a * z[q]);
    out[k + Mh] = 2.0 / (w * J);
  }
}

}  // namespace spf
